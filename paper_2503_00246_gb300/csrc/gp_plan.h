// Host-side plan of the ghost-penalty operator: classification, face list,
// active-DoF numbering, 1D reference matrices and the tables the kernels read.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "gp.h"

namespace gp {

constexpr int KMAX = 8;
constexpr int ZRUN_MAX = 256;       // elements per zero run (one CTA pass)
// ints per brick descriptor: first local cell, own cells, local cells, first face, faces,
// brick coordinates bx, by, bz, first face of axis 1 and of axis 2 (the faces are sorted by axis)
constexpr int BDESC = 10;
constexpr int SLAB = 8;             // ints per slab of the slab pipeline

enum : int8_t { OUTSIDE = 0, CUT = 1, INSIDE = 2 };

struct Plan {
  int dim = 0, n = 0, k = 0, precision = GP_FP64;
  double lo[3] = {0, 0, 0};
  double h = 0;
  int nl = 0;                     // lattice nodes per axis, n*k+1
  int64_t ncell = 0;              // n^dim
  int64_t nrows = 0;              // lattice rows along x, nl^(dim-1)
  int L = 0;                      // tangential nodes per face, (k+1)^(dim-1)

  std::vector<int8_t> cls;        // cell classes, lexicographic (x fastest)
  int64_t cell_counts[3] = {0, 0, 0};

  // ghost faces, sorted by normal axis then lower cell
  int32_t fstart[4] = {0, 0, 0, 0};
  std::vector<int64_t> face_cell; // lower cell (lexicographic index)
  std::vector<int32_t> face_inv;  // 2 per face: involved-cell index of K-, K+
  std::vector<int64_t> inv_cells; // involved cells (sorted)
  std::vector<int32_t> rowtab;    // ninv x L: compact index of (ci*k, row tau) per involved cell
  // per-face row starts of the patch: axis 0: L rows (one per normal line, 2k+1 long);
  // axis a > 0: (2k+1)*(k+1)^(d-2) rows (normal index b, outer tangential index), k+1 long
  std::vector<int32_t> frows;
  int64_t rbase[4] = {0, 0, 0, 0};
  std::vector<int32_t> face_of;   // dim x ncell: face id of (axis, lower cell), -1 if none

  // active-DoF numbering: per lattice row, active x-runs and the compact start
  int64_t n_active = 0, n_touched = 0;
  std::vector<int64_t> row_start; // nrows
  std::vector<int32_t> run_off;   // nrows+1, offsets into runs
  std::vector<int32_t> runs;      // (X0, X1) inclusive pairs

  // lift work: owner cells (ci, cj, cl, 0) with coordinates in [0, n], sorted by the
  // pattern of faces whose patch reaches them; lrow[cell][row] is the compact index of
  // node (ci*k, cj*k+q, cl*k+r), row = q + k r, or -1 if that node is inactive
  std::vector<int32_t> lcell;
  std::vector<int32_t> lrow;
  std::vector<int32_t> lwin;      // nlift x (3*12 | 2*6): candidate face ids (-1 if none)
  int lwin_width = 0;
  // zero fill of the active DoFs outside every face patch: runs (c0, len <= 256)
  std::vector<int32_t> zruns;
  int64_t num_lift_cells() const { return (int64_t)lcell.size() / 4; }
  int64_t num_zero_runs() const { return (int64_t)zruns.size() / 2; }

  // active cells for the mass + stiffness operator (lexicographic)
  std::vector<int32_t> crow;      // ncact x (k+1)^(d-1): compact index of (ci k, cj k + q, cl k + r)
  int64_t num_active_cells() const { return ncact; }
  int64_t ncact = 0;
  // owner cells of the active nodes (coordinates in [0, n]; those a ghost face reaches first,
  // in lift order, then the rest lexicographic): per owner the
  // active-cell index of the 2^d cells (ci - s_x, cj - s_y, cl - s_z) (-1 if none), and per
  // x-row (q, r) the compact index of node (ci k, cj k + q, cl k + r) ([ncown][KR], -1 if none)
  std::vector<int32_t> cwin;
  std::vector<int32_t> corow;
  std::vector<int64_t> cown;      // owner cells: linear index ci + (n+1) (cj + (n+1) cl)
  int64_t ncown = 0;

  // slab partition (Sec. 2.7): cell layers [part_lo, part_hi) along the last axis.  The
  // vector is the global numbering restricted to the lattice planes [part_lo k,
  // min(part_hi + 1, n) k] of that axis: entries [0, n_owned) are owned, the rest is the
  // one-cell halo above; the first n_lower entries are the halo of the partition below.
  bool partitioned = false;
  int part_lo = 0, part_hi = 0;
  int64_t n_global = 0, g_offset = 0, n_owned = 0, n_lower = 0;

  // brick path (build_bricks): the mesh cut into bricks of bdim cells; one CTA per non-empty
  // brick stages the cell blocks of its involved cells, evaluates every ghost face with a cell
  // in the brick, accumulates per-cell outputs and writes its nodes (see gp_brick.cuh)
  int bdim[3] = {0, 0, 0};        // cells per brick along each axis; bdim[0] == 0: no brick path
  int nbx[3] = {1, 1, 1};         // bricks per axis
  std::vector<int32_t> bdesc;     // BDESC ints per non-empty brick (see gp_brick.cuh)
  std::vector<int32_t> bcell;     // per brick: involved-cell indices, own cells first, then halo cells
  std::vector<int32_t> bccoord;   // parallel to bcell: packed local coords cx | cy << 8 | cz << 16 (own)
  std::vector<uint32_t> bface;    // per brick: packed faces (axis, local K-, local K+, own flags)
  std::vector<int32_t> bslot;     // dense brick index -> non-empty brick slot, or -1
  std::vector<int32_t> pnode;     // per plane node: compact index of the DoF
  std::vector<int32_t> poff;      // plane nodes + 1: CSR offsets into pslot
  std::vector<int32_t> pslot;     // per plane node, in increasing brick index: the partial-grid
                                  // entry of each brick holding an involved cell that contains it
  int64_t pgrid = 0;              // partial-grid entries per brick slot
  int32_t goff[3][2] = {{0, 0}, {0, 0}, {0, 0}};  // box face (axis, side) offset in a brick's grid
  int32_t gstride[3] = {0, 0, 0};                 // row stride of box face a's grid
  int bmax_own = 0, bmax_cell = 0, bmax_face = 0;
  int64_t num_bricks() const { return bdim[0] == 0 ? 0 : (int64_t)bdesc.size() / BDESC; }

  // slab pipeline of the face + lift path (build_slabs): SLAB ints per slab, the owner range
  // [lo, hi) of the lift, then per axis the face range [lo, hi) that the slab's face launch
  // evaluates (axes >= dim: 0, 0)
  std::vector<int32_t> slabs;
  int num_slabs() const { return (int)(slabs.size() / SLAB); }
  int64_t num_plane_nodes() const { return (int64_t)pnode.size(); }

  // FP64 1D reference data
  std::vector<double> gl;         // k+1 Gauss-Lobatto points on [0,1]
  std::vector<double> stiff;      // (k+1)^2: int_0^1 l_a' l_b' 
  std::vector<double> mass;       // (k+1)^2
  std::vector<double> jumps;      // k x (2k+1)
  std::vector<double> scale;      // k: c_j h^(dim-2) (macro patch: gamma lambda_j h^dim)
  int stabilization = GP_STAB_GHOST;

  int64_t num_faces() const { return (int64_t)face_cell.size(); }
  int64_t compact(int X, int64_t row) const;
};

inline int64_t ipow_host(int64_t b, int e) {
  int64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}

gp_status build_plan(const gp_mesh* mesh, const gp_levelset* ls, const gp_opts* opts,
                     Plan& p, std::string& err);
void active_coords(const Plan& p, double* xyz);
// Weighted slab partition of the cell layers along the last axis into nparts pieces;
// bounds receives nparts + 1 layer indices.
gp_status partition_slabs(const gp_mesh* mesh, const gp_levelset* ls, const gp_opts* opts, int nparts,
                          int32_t* bounds, std::string& err);

// 1D precompute (exposed for the unit tests through gp_reference_1d)
void gauss_lobatto_01(int k, std::vector<double>& x);
void reference_1d(int k, const std::vector<double>& gl, std::vector<double>& mass,
                  std::vector<double>& jumps);
void reference_stiffness(int k, std::vector<double>& stiff);
// Macro-patch 1D data: k mirror-(anti)symmetric vectors (k x (2k+1)) and weights lambda_j;
// false if the matrix is not of rank k with the expected parities.
bool macro_patch_1d(int k, std::vector<double>& vecs, std::vector<double>& lambda);
// Brick tables for the fused face + lift kernel: picks the brick shape (largest first) whose
// staged cell blocks, per-cell outputs and row starts fit smem_budget bytes of shared memory
// with values of vbytes and accumulators of sbytes bytes (extra: the bytes of the jump planes
// of one chunk of faces), and fills bdim, nbx, bdesc, bcell, bccoord, bface, bslot, pnode,
// poff, pslot, pgrid, goff and gstride.  Returns false (bdim[0] = 0) when no shape fits.
bool build_bricks(Plan& p, int vbytes, int sbytes, size_t extra, size_t smem_budget);
// Slab pipeline of the face + lift path: cuts the lift owners (lexicographic, or sorted within
// groups of SLAB_GROUP) into about nslab ranges of whole groups, and gives each range the faces
// of each axis that it needs and no earlier range needed (the faces of an axis follow the
// lexicographic order of their lower cells, as the owners do, so each is an id range).  The last
// range also takes the remaining faces.  Fills slabs; nslab <= 1, or fewer than two ranges: empty.
constexpr int SLAB_GROUP = 256;
std::vector<int32_t> slab_table(const Plan& p, int nslab);
void build_slabs(Plan& p, int nslab);   // p.slabs = slab_table(p, nslab)
// For a slab table of ns slabs: ns + 1 compact indices b, b[0] = 0, b[ns] = n_active, such that
// the entries [b[s], b[s + 1]) of y are final once slabs 0..s are lifted (and the zero fill done).
std::vector<int64_t> slab_y_bounds(const Plan& p, const std::vector<int32_t>& table);
// For a slab table of ns slabs: ns compact indices b, b[s] = one past the largest index of x the
// face launches of slabs 0..s read.
std::vector<int64_t> slab_x_bounds(const Plan& p, const std::vector<int32_t>& table);
// Builds crow, cwin and corow (the tables of the mass + stiffness operator).
void build_cell_table(Plan& p);
// For each owner cell of `cells` (same mesh), its index in the lift owner list of `faces`
// (-1 if no ghost face reaches it): the fused gather of the model system uses it.
std::vector<int32_t> owner_lift_index(const Plan& cells, const Plan& faces);
// Every index of the cell table inside the active DoFs and the active cells.
bool check_cell_table(const Plan& p);
// diag(M_active + K_active + G) in FP64 (needs the cell table).
void build_diagonal(const Plan& p, std::vector<double>& diag);

}  // namespace gp
