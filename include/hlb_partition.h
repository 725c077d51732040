/*
 * hlb_partition.h — domain decomposition of a sparse lattice and the halo
 * exchange between its parts (part of libhemegb).
 *
 * The paper runs one MPI rank per GPU (arXiv 2202.11770, Section 3.1): the
 * lattice is split into domains, each rank steps its own sites, and the
 * populations that stream across a domain edge are exchanged every step; on
 * the GPU the received populations are scattered into the local arrays
 * (Section 3.2.2, the GPU_StreamReceivedDistr kernel) and the edge exchange is
 * ordered to overlap with the interior computation (Section 3.2.3).
 *
 * Here a part is a contiguous range of the (z, y, x)-ordered site list
 * ("slab"), cut into equal site counts.  Its local lattice holds its own
 * ("owned") sites and a ghost copy of every remote site that an owned site
 * pulls from, all in global order, so that each part is an ordinary lattice
 * for hlb_create (its compact index table still fits).  A ghost's own links
 * that leave the local lattice, and its iolet links, become wall links: a
 * ghost's values are never read before the exchange overwrites them.
 *
 * A partitioned run steps every part with the pull A-B scheme and then, for
 * every pair (q, p), copies the post-collision populations s'_i(y) that the
 * owned sites of p pull from q's site y into the ghost slot of y in p
 * (hlb_halo_pack on q, transport, hlb_halo_unpack on p).  The owned sites of
 * every part then see exactly the inputs of the undivided lattice: their
 * states are bit-identical to the undivided run.
 *
 * Slot numbers address a population array [19][n_local] (element i * n_local
 * + site).  All arrays returned are owned by the plan and valid until
 * hlb_part_destroy.  Errors as in hemegb.h (HLB_ERR_ARG for a bad argument,
 * HLB_ERR_NOMEM when a host allocation fails).
 */
#ifndef HLB_PARTITION_H
#define HLB_PARTITION_H

#include <stdint.h>

#include "hemegb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hlb_part hlb_part;

/* Plan the split of `lat` (as accepted by hlb_create) into n_parts slabs of
 * equal site counts (1 <= n_parts <= n_sites). */
int hlb_part_create(const hlb_lattice* lat, int32_t n_parts, hlb_part** out);
int hlb_part_destroy(hlb_part* plan);
int32_t hlb_part_count(const hlb_part* plan);

/* Local lattice of part p (arrays owned by the plan; iolets as in the global
 * lattice), its owned sites [owned_lo, owned_hi) in local indexing, and the
 * global index of every local site (global[n_local], ascending). */
int hlb_part_local(const hlb_part* plan, int32_t p, hlb_lattice* local, int64_t* owned_lo, int64_t* owned_hi,
                   const int64_t** global);

/* Post-collision exchange from part q to part p (q != p): n slots of q's
 * population array (src) and the matching slots of p's (dst), in the same
 * order; n = 0 when p pulls nothing from q. */
int hlb_part_halo(const hlb_part* plan, int32_t q, int32_t p, int64_t* n, const int64_t** src_slots,
                  const int64_t** dst_slots);

/* Ghost sites of p owned by q: n local sites of q and the matching local sites
 * of p (whole-site copies, for solvers that exchange pre-collision states). */
int hlb_part_ghosts(const hlb_part* plan, int32_t q, int32_t p, int64_t* n, const int64_t** src_sites,
                    const int64_t** dst_sites);

/* Device side, on the solver's stream, asynchronously.  slots: int64 [n] in
 * device memory; buf: n elements of the solver's storage precision in device
 * memory.  pack gathers buf[k] = f[slots[k]] from the post-collision state
 * that the solver's next step gathers from; unpack scatters it back.  Both
 * need a pull A-B solver that has stepped (HLB_ERR_STATE otherwise). */
int hlb_halo_pack(hlb_solver* h, const int64_t* slots, int64_t n, void* buf);
int hlb_halo_unpack(hlb_solver* h, const int64_t* slots, int64_t n, const void* buf);

/* Part of one pull A-B step (after the solver's first step), for the edge-
 * first order of a partitioned run (Section 3.2.3): the step of the sites in
 * the 256-site tiles [first_tile, first_tile + n_tiles) and, with
 * iolet_sites != 0, of the sites with iolet links.  The ranges of one step
 * must cover every tile once and the iolet sites once; the call with
 * finish != 0, the last of the step, advances the solver to the next time.
 * Launches in stream order on the solver's stream; between the calls the
 * caller may pack the halo of the tiles already stepped (hlb_set_stream
 * moves the solver to another stream); hlb_halo_pack and hlb_halo_unpack
 * then address the state being written.  Until the finishing call, no other
 * call reads or steps the solver (hlb_step returns HLB_ERR_STATE).
 * HLB_ERR_STATE for an AA solver, before the first step, or with Windkessel
 * outlets. */
int hlb_step_range(hlb_solver* h, int64_t first_tile, int64_t n_tiles, int32_t iolet_sites, int32_t finish);

/* Restrict the total mass of hlb_reduce to the local sites [lo, hi): a
 * part's owned sites.  The iolet fluxes need no restriction (ghosts carry no
 * iolet links).  A new solver counts all its sites. */
int hlb_set_owned_range(hlb_solver* h, int64_t lo, int64_t hi);

#ifdef __cplusplus
}
#endif
#endif
