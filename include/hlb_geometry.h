/*
 * hlb_geometry.h — seeded synthetic sparse lattices (input generator).
 *
 * This library builds the inputs that both the FP64 oracle and the GPU solver
 * consume: a list of fluid sites on an integer lattice, the D3Q19 pull-source
 * table with wall / iolet link codes, per-site types, analytic wall normals,
 * amplitude groups of velocity-iolet sites and the iolet descriptors.  It
 * holds none of the lattice Boltzmann arithmetic (no equilibrium, collision,
 * streaming or boundary values); it only voxelises geometry.
 *
 * Paper context (arXiv 2202.11770):
 *   - Section 3.2.1: the GPU code is initialised from a pre-processed sparse
 *     geometry: streaming indices, wall/iolet link information, iolet site
 *     ranges and iolet normals.  This library produces the equivalent inputs.
 *   - Section 3.2.2: fluid sites fall into six collision-streaming types
 *     (inner, wall, inlet, outlet, inlet+wall, outlet+wall); hlbg_type()
 *     reports them.
 *   - Section 2.2: D3Q19 velocity set.  Direction order used throughout:
 *       0: (0,0,0)
 *       1..6:  (+1,0,0) (-1,0,0) (0,+1,0) (0,-1,0) (0,0,+1) (0,0,-1)
 *       7..18: (+1,+1,0) (-1,-1,0) (+1,-1,0) (-1,+1,0) (+1,0,+1) (-1,0,-1)
 *              (+1,0,-1) (-1,0,+1) (0,+1,+1) (0,-1,-1) (0,+1,-1) (0,-1,+1)
 *     so the opposite of direction i >= 1 is i+1 (i odd) or i-1 (i even).
 *
 * Layouts (all arrays owned by the lattice object, valid until hlbg_free):
 *   xyz[n][3]        int32, site coordinates, row-major (x,y,z per site).
 *   src[18][n]       int32, SoA.  src[(i-1)*n + s] for direction i = 1..18 is
 *                    the index of the fluid site at x_s - c_i, or a link code:
 *                    -1 = wall link, -(2+k) = link through iolet k.
 *   type[n]          uint8, HLBG_INNER .. HLBG_OUTLET_WALL.
 *   wall_normal[3][n] float, SoA; unit normal pointing into the fluid at sites
 *                    with at least one wall link, 0 elsewhere.
 *   amp_group[n]     int32; for sites with a link through a velocity iolet,
 *                    the iolet-local amplitude group (0..n_groups-1); 0
 *                    elsewhere.
 * Sites are ordered lexicographically by (z, y, x).
 *
 * Link classification: a link from fluid site x along c_i whose end x+c_i is
 * not fluid is an iolet-k link when its midpoint m = x + c_i/2 lies in the
 * slab -1 <= (m - centre_k).normal_k <= 0 (on or beyond the iolet plane, the
 * normal pointing into the fluid) and within radius_k of the iolet axis;
 * otherwise it is a wall link.
 *
 * Errors: every function returning int gives 0 on success and a negative
 * value on failure; hlbg_last_error() then returns a message (thread-local).
 */
#ifndef HLB_GEOMETRY_H
#define HLB_GEOMETRY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { HLBG_INNER = 0, HLBG_WALL = 1, HLBG_INLET = 2, HLBG_OUTLET = 3,
       HLBG_INLET_WALL = 4, HLBG_OUTLET_WALL = 5 };
/* End treatment of a pipe end / kind of an iolet. */
enum { HLBG_END_VELOCITY = 0, HLBG_END_PRESSURE = 1, HLBG_END_WALL = 2 };

typedef struct {
  int32_t kind;       /* HLBG_END_VELOCITY or HLBG_END_PRESSURE            */
  int32_t role;       /* 0 = inlet, 1 = outlet (site types only)           */
  double centre[3];   /* a point on the iolet plane, on the vessel axis    */
  double normal[3];   /* unit normal of the plane, pointing into the fluid */
  double radius;      /* vessel radius at the iolet                        */
  int32_t n_groups;   /* amplitude groups (velocity iolets), >= 1          */
} hlbg_iolet;

typedef struct hlbg_lattice hlbg_lattice;

/* Straight pipe along +z: sites with x^2 + y^2 < radius^2 (integer x, y,
 * axis through the origin) and z = 0 .. length-1.  The ends are the planes
 * z = -1/2 (inlet, normal +z) and z = length-1/2 (outlet, normal -z); each is
 * a velocity iolet, a pressure iolet or closed by walls (HLBG_END_*).  Iolets
 * are numbered in the order inlet, outlet, skipping walled ends.
 * radius 8, length 64 gives 12,352 sites. */
int hlbg_pipe(double radius, int32_t length, int32_t inlet_kind,
              int32_t outlet_kind, hlbg_lattice** out);

/* Seeded bifurcating tree: a binary tree of `depth` bifurcation levels
 * (2^depth leaves) of straight capsule segments, radii shrinking by Murray's
 * law r_child = r_parent / 2^(1/3), segment length = length_ratio * radius,
 * full bifurcation angle uniform in [30, 70] degrees, bifurcation plane turned
 * 90 +- 20 degrees about each daughter axis.  The root starts on the plane
 * z = -1/2 along +z with its axis on x = y = 0 and a flat velocity inlet;
 * every leaf ends in a flat pressure outlet.  If target_sites > 0 the root
 * radius is chosen by iteration so that the site count is within 2 % of it;
 * otherwise root_radius is used as given.  The velocity inlet's sites are
 * split into n_sectors angular sectors x n_rings equal-area rings
 * (group = ring * n_sectors + sector).  A shape whose outlet planes are
 * crossed by another segment is rejected and redrawn from the same stream. */
int hlbg_tree(int32_t depth, uint64_t seed, int64_t target_sites,
              double root_radius, double length_ratio, int32_t n_sectors,
              int32_t n_rings, hlbg_lattice** out);

int64_t hlbg_n_sites(const hlbg_lattice* L);
const int32_t* hlbg_xyz(const hlbg_lattice* L);
const int32_t* hlbg_src(const hlbg_lattice* L);
const uint8_t* hlbg_type(const hlbg_lattice* L);
const float* hlbg_wall_normal(const hlbg_lattice* L);
const int32_t* hlbg_amp_group(const hlbg_lattice* L);
int32_t hlbg_n_iolets(const hlbg_lattice* L);
const hlbg_iolet* hlbg_iolets(const hlbg_lattice* L);
/* info[0] root radius, info[1] bounding-box fill fraction, info[2..4]
 * bounding-box extent (x, y, z), info[5] number of segments, info[6] number of
 * shapes rejected before this one, info[7] root segment length. */
void hlbg_info(const hlbg_lattice* L, double info[8]);
void hlbg_free(hlbg_lattice* L);
const char* hlbg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
