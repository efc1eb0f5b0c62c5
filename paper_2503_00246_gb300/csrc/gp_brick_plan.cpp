// Host tables of the brick path: bricks of cells, their involved cells and faces, the plane
// nodes shared by several bricks (see gp_brick.cuh for the kernels that read them).
#include <algorithm>
#include <cstring>

#include "gp_plan.h"

namespace gp {

namespace {

// packed face record: axis (bits 0-1), local K- (2-11), local K+ (12-21), K- own (22), K+ own (23)
uint32_t pack_face(int axis, int lo, int hi, bool lo_own, bool hi_own) {
  return (uint32_t)axis | ((uint32_t)lo << 2) | ((uint32_t)hi << 12) | ((uint32_t)lo_own << 22) |
         ((uint32_t)hi_own << 23);
}

struct BrickShape {
  int b[3];
};

// partial-grid entries of one brick: for every axis a and side, one value per node of the
// box face, (b_u k + 1) nodes along each other axis u
int64_t grid_entries(int d, const int b[3], int k) {
  int64_t tot = 0;
  for (int a = 0; a < d; ++a) {
    int64_t e = 1;
    for (int u = 0; u < d; ++u)
      if (u != a) e *= (int64_t)b[u] * k + 1;
    tot += 2 * e;
  }
  return tot;
}

}  // namespace

bool build_bricks(Plan& p, int vbytes, int sbytes, size_t extra, size_t smem_budget) {
  const int d = p.dim, n = p.n, k = p.k, L = p.L;
  p.bdim[0] = p.bdim[1] = p.bdim[2] = 0;
  p.bdesc.clear();
  p.bcell.clear();
  p.bccoord.clear();
  p.bface.clear();
  p.bslot.clear();
  p.pnode.clear();
  p.poff.clear();
  p.pslot.clear();
  const int64_t nf = p.num_faces();
  if (nf == 0 || p.partitioned) return false;
  static const BrickShape shapes3[4] = {{{4, 4, 4}}, {{4, 4, 2}}, {{4, 2, 2}}, {{2, 2, 2}}};
  static const BrickShape shapes2[4] = {{{16, 16, 1}}, {{8, 8, 1}}, {{4, 4, 1}}, {{2, 2, 1}}};
  const BrickShape* shapes = d == 3 ? shapes3 : shapes2;
  constexpr size_t nshapes = 4;
  const int64_t stride[3] = {1, n, (int64_t)n * n};
  auto coords = [&](int64_t c, int out[3]) {
    out[0] = (int)(c % n);
    out[1] = (int)((c / n) % n);
    out[2] = d == 3 ? (int)(c / ((int64_t)n * n)) : 0;
  };
  std::vector<int32_t> inv_of(p.ncell, -1);
  for (size_t i = 0; i < p.inv_cells.size(); ++i) inv_of[p.inv_cells[i]] = (int32_t)i;
  const int64_t nbl = ipow_host(k + 1, d);
  // pick the largest shape whose busiest brick fits the budget
  for (size_t si = 0; si < nshapes; ++si) {
    const int* B = shapes[si].b;
    int nbx[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) nbx[a] = (n + B[a] - 1) / B[a];
    const int64_t ndense = (int64_t)nbx[0] * nbx[1] * nbx[2];
    auto brick_of = [&](int64_t c) -> int64_t {
      int cc[3];
      coords(c, cc);
      return (cc[0] / B[0]) + (int64_t)nbx[0] * ((cc[1] / B[1]) + (int64_t)nbx[1] * (cc[2] / B[2]));
    };
    // faces per brick (a face belongs to the brick of each of its two cells), in face order
    std::vector<std::vector<int32_t>> faces_of(ndense);
    for (int a = 0; a < d; ++a)
      for (int64_t f = p.fstart[a]; f < p.fstart[a + 1]; ++f) {
        const int64_t c0 = p.face_cell[f], c1 = c0 + stride[a];
        const int64_t b0 = brick_of(c0), b1 = brick_of(c1);
        faces_of[b0].push_back((int32_t)f);
        if (b1 != b0) faces_of[b1].push_back((int32_t)f);
      }
    // per brick: own involved cells (lexicographic), halo cells (sorted)
    std::vector<std::vector<int64_t>> own(ndense);
    for (int64_t c : p.inv_cells) own[brick_of(c)].push_back(c);   // inv_cells is sorted
    int max_own = 0, max_cell = 0, max_face = 0;
    std::vector<std::vector<int64_t>> halo(ndense);
    for (int64_t b = 0; b < ndense; ++b) {
      if (faces_of[b].empty()) continue;
      for (int32_t f : faces_of[b]) {
        int a = 0;
        while (f >= p.fstart[a + 1]) ++a;
        const int64_t c0 = p.face_cell[f], c1 = c0 + stride[a];
        if (brick_of(c0) != b) halo[b].push_back(c0);
        if (brick_of(c1) != b) halo[b].push_back(c1);
      }
      std::sort(halo[b].begin(), halo[b].end());
      halo[b].erase(std::unique(halo[b].begin(), halo[b].end()), halo[b].end());
      max_own = std::max(max_own, (int)own[b].size());
      max_cell = std::max(max_cell, (int)(own[b].size() + halo[b].size()));
      max_face = std::max(max_face, (int)faces_of[b].size());
    }
    // the kernel's layout: accumulators, x blocks, own coordinates, then one region for either
    // the local row starts or the jump planes (extra bytes), each rounded up to 16 bytes
    const size_t need = (size_t)max_cell * nbl * vbytes + (size_t)max_own * nbl * sbytes + (size_t)max_own * 4 +
                        std::max(extra, (size_t)max_cell * L * 4) + 48;
    const bool last = si + 1 == nshapes;
    if (max_cell >= 1024 || (need > smem_budget && !last)) continue;
    if (need > smem_budget) return false;
    // ---- commit this shape
    for (int a = 0; a < 3; ++a) {
      p.bdim[a] = a < d ? B[a] : 1;
      p.nbx[a] = nbx[a];
    }
    p.bmax_own = max_own;
    p.bmax_cell = max_cell;
    p.bmax_face = max_face;
    p.pgrid = grid_entries(d, B, k);
    p.bslot.assign(ndense, -1);
    int32_t slot = 0;
    for (int64_t b = 0; b < ndense; ++b) {
      if (faces_of[b].empty()) continue;
      p.bslot[b] = slot++;
      const int bx = (int)(b % nbx[0]), by = (int)((b / nbx[0]) % nbx[1]), bz = (int)(b / ((int64_t)nbx[0] * nbx[1]));
      const int32_t cell_off = (int32_t)p.bcell.size(), face_off = (int32_t)p.bface.size();
      std::vector<int64_t> loc(own[b]);
      loc.insert(loc.end(), halo[b].begin(), halo[b].end());
      for (size_t i = 0; i < loc.size(); ++i) {
        p.bcell.push_back(inv_of[loc[i]]);
        int cc[3];
        coords(loc[i], cc);
        const bool is_own = i < own[b].size();
        p.bccoord.push_back(is_own ? ((cc[0] - bx * B[0]) | ((cc[1] - by * B[1]) << 8) | ((cc[2] - bz * B[2]) << 16))
                                   : -1);
      }
      auto local = [&](int64_t c) -> int {
        return (int)(std::lower_bound(loc.begin(), loc.begin() + own[b].size(), c) - loc.begin());
      };
      auto local_any = [&](int64_t c, bool& is_own) -> int {
        auto it = std::lower_bound(loc.begin(), loc.begin() + own[b].size(), c);
        if (it != loc.begin() + own[b].size() && *it == c) {
          is_own = true;
          return (int)(it - loc.begin());
        }
        is_own = false;
        auto h = std::lower_bound(loc.begin() + own[b].size(), loc.end(), c);
        return (int)(h - loc.begin());
      };
      (void)local;
      for (int32_t f : faces_of[b]) {
        int a = 0;
        while (f >= p.fstart[a + 1]) ++a;
        const int64_t c0 = p.face_cell[f], c1 = c0 + stride[a];
        bool o0 = false, o1 = false;
        const int l0 = local_any(c0, o0), l1 = local_any(c1, o1);
        p.bface.push_back(pack_face(a, l0, l1, o0, o1));
      }
      int32_t astart[3] = {0, 0, 0};   // first face of each axis within the brick's list
      for (int a = 1; a < 3; ++a) {
        astart[a] = astart[a - 1];
        while (astart[a] < (int32_t)faces_of[b].size() && faces_of[b][astart[a]] < p.fstart[a]) ++astart[a];
      }
      const int32_t desc[BDESC] = {cell_off, (int32_t)own[b].size(), (int32_t)loc.size(), face_off,
                                   (int32_t)faces_of[b].size(), bx, by, bz, astart[1], astart[2]};
      p.bdesc.insert(p.bdesc.end(), desc, desc + BDESC);
    }
    break;
  }
  if (p.bdim[0] == 0) return false;
  // ---- partial grids of a brick: for axis a and side (0 lower, 1 upper) one entry per node of
  // the box face, rows along the first other axis u0 (bdim[u0] k + 1 entries each)
  {
    int32_t off = 0;
    for (int a = 0; a < 3; ++a) {
      const int u0 = a == 0 ? 1 : 0, u1 = a == 2 ? 1 : 2;
      p.gstride[a] = p.bdim[u0] * k + 1;
      const int32_t e = a < d ? (p.bdim[u0] * k + 1) * (d == 3 ? p.bdim[u1] * k + 1 : 1) : 0;
      for (int side = 0; side < 2; ++side) {
        p.goff[a][side] = off;
        off += e;
      }
    }
    if (off != p.pgrid) { p.bdim[0] = 0; return false; }
  }
  std::vector<uint8_t> invmask(p.ncell, 0);
  for (int64_t c : p.inv_cells) invmask[c] = 1;
  const int64_t nl = p.nl;
  const int64_t nnodes = ipow_host(nl, d);
  std::vector<uint8_t> seen(nnodes, 0);
  for (int64_t c : p.inv_cells) {
    int cc[3];
    coords(c, cc);
    const int zr = d == 3 ? k : 0;
    for (int r = 0; r <= zr; ++r)
      for (int q = 0; q <= k; ++q)
        for (int pp = 0; pp <= k; ++pp) {
          const int X[3] = {cc[0] * k + pp, cc[1] * k + q, cc[2] * k + r};
          bool plane = false;
          for (int a = 0; a < d; ++a) {
            const int pk = p.bdim[a] * k;
            if (X[a] % pk == 0 && X[a] > 0 && X[a] < n * k) plane = true;
          }
          if (!plane) continue;
          const int64_t lin = X[0] + nl * (X[1] + (d == 3 ? nl * X[2] : 0));
          if (seen[lin]) continue;
          seen[lin] = 1;
        }
  }
  // per plane node: the partial-grid entries of the bricks that hold an involved cell containing
  // it, in increasing brick index (the order in which the fixup adds them); the entry of a brick
  // is on its box face of the lowest axis on which the node lies on an inner brick boundary
  p.poff.assign(1, 0);
  for (int64_t lin = 0; lin < nnodes; ++lin) {
    if (!seen[lin]) continue;
    const int X[3] = {(int)(lin % nl), (int)((lin / nl) % nl), d == 3 ? (int)(lin / (nl * nl)) : 0};
    const int64_t row = X[1] + (d == 3 ? nl * X[2] : 0);
    const int64_t ci = p.compact(X[0], row);
    if (ci < 0) { p.bdim[0] = 0; return false; }
    int c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0}, pa = -1;
    for (int a = 0; a < d; ++a) {
      const bool on = X[a] % k == 0;
      c0[a] = on ? std::max(X[a] / k - 1, 0) : X[a] / k;
      c1[a] = on ? std::min(X[a] / k, n - 1) : X[a] / k;
      if (pa < 0 && X[a] % (p.bdim[a] * k) == 0 && X[a] > 0 && X[a] < n * k) pa = a;
    }
    const int u0 = pa == 0 ? 1 : 0, u1 = pa == 2 ? 1 : 2;
    for (int bz = c0[2] / p.bdim[2]; bz <= c1[2] / p.bdim[2]; ++bz)
      for (int by = c0[1] / p.bdim[1]; by <= c1[1] / p.bdim[1]; ++by)
        for (int bx = c0[0] / p.bdim[0]; bx <= c1[0] / p.bdim[0]; ++bx) {
          const int bb[3] = {bx, by, bz};
          bool found = false;
          for (int cz = c0[2]; cz <= c1[2]; ++cz)
            for (int cy = c0[1]; cy <= c1[1]; ++cy)
              for (int cx = c0[0]; cx <= c1[0]; ++cx)
                if (cx / p.bdim[0] == bx && cy / p.bdim[1] == by && cz / p.bdim[2] == bz &&
                    invmask[cx + (int64_t)n * (cy + (int64_t)(d == 3 ? n : 0) * cz)])
                  found = true;
          if (!found) continue;
          const int32_t slot = p.bslot[bx + (int64_t)p.nbx[0] * (by + (int64_t)p.nbx[1] * bz)];
          if (slot < 0) { p.bdim[0] = 0; return false; }
          const int side = X[pa] == bb[pa] * p.bdim[pa] * k ? 0 : 1;
          const int64_t g = (X[u0] - bb[u0] * p.bdim[u0] * k) +
                            (d == 3 ? (int64_t)p.gstride[pa] * (X[u1] - bb[u1] * p.bdim[u1] * k) : 0);
          const int64_t e = (int64_t)slot * p.pgrid + p.goff[pa][side] + g;
          if (e < 0 || e >= (int64_t)(p.bdesc.size() / BDESC) * p.pgrid || e >= ((int64_t)1 << 31)) {
            p.bdim[0] = 0;
            return false;
          }
          p.pslot.push_back((int32_t)e);
        }
    p.pnode.push_back((int32_t)ci);
    p.poff.push_back((int32_t)p.pslot.size());
  }
  // ---- bounds of every index the brick kernels read or write
  const int64_t ninv = (int64_t)p.inv_cells.size();
  for (int32_t i : p.bcell)
    if (i < 0 || i >= ninv) { p.bdim[0] = 0; return false; }
  for (size_t i = 0; i < p.rowtab.size(); ++i)
    if (p.rowtab[i] < 0 || p.rowtab[i] + k + 1 > p.n_active) { p.bdim[0] = 0; return false; }
  return true;
}

}  // namespace gp
