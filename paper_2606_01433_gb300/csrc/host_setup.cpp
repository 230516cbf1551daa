// Host symbolic setup: dof numbering, sparsity patterns, overlapping subdomains, slab
// orderings of the local problems, interface entities and the coarse-space index maps of
// every level (arXiv 2606.01433, Section 2.1 and Section 2.2).  No floating-point
// arithmetic of the method happens here; the device does all numeric work.
#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <thread>

#include <atomic>
#include <cmath>

#include "common.h"

namespace gdsw {

// ------------------------------------------------------------------ small utilities
template <typename F>
static void parallel_for(int64_t n, F f) {
  int nt = int(std::thread::hardware_concurrency());
  if (nt < 1) nt = 1;
  if (nt > 32) nt = 32;
  if (n < 4096 || nt == 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    int64_t a = t * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    th.emplace_back([=] {
      for (int64_t i = a; i < b; ++i) f(i);
    });
  }
  for (auto& x : th) x.join();
}

// n independent tasks of uneven size (one per part): dynamic scheduling over the threads
template <typename F>
static void parallel_tasks(int64_t n, F f) {
  int nt = int(std::thread::hardware_concurrency());
  nt = std::max(1, std::min<int>(nt, 32));
  if (n <= 1 || nt == 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < std::min<int64_t>(nt, n); ++t)
    th.emplace_back([&] {
      for (int64_t i = next++; i < n; i = next++) f(i);
    });
  for (auto& x : th) x.join();
}

// elements (per axis) containing node coordinate c on an axis with n elements
static inline int elem_range(int c, int n, int* e) {
  int cnt = 0;
  if (c % 2 == 0) {
    if (c / 2 - 1 >= 0) e[cnt++] = c / 2 - 1;
    if (c / 2 < n) e[cnt++] = c / 2;
  } else {
    e[cnt++] = c / 2;
  }
  return cnt;
}

bool MeshHost::shares_element(int64_t a, int64_t b) const {
  int ia, ja, ka, ib, jb, kb;
  coords(a, ia, ja, ka);
  coords(b, ib, jb, kb);
  int lo[3] = {std::max(ia, ib), std::max(ja, jb), std::max(ka, kb)};
  int hi[3] = {std::min(ia, ib), std::min(ja, jb), std::min(ka, kb)};
  int nn[3] = {nx, ny, nz};
  int e0[3], e1[3];
  for (int d = 0; d < 3; ++d) {
    if (lo[d] - hi[d] > 2) return false;
    // element e contains both iff 2e <= hi and 2e + 2 >= lo
    e0[d] = std::max(0, (lo[d] - 1) / 2);  // ceil((lo-2)/2) for lo >= 0
    if (lo[d] < 2) e0[d] = 0;
    e1[d] = std::min(nn[d] - 1, hi[d] / 2);
    if (e0[d] > e1[d]) return false;
  }
  for (int ez = e0[2]; ez <= e1[2]; ++ez)
    for (int ey = e0[1]; ey <= e1[1]; ++ey)
      for (int ex = e0[0]; ex <= e1[0]; ++ex)
        if (mask[ex + int64_t(nx) * (ey + int64_t(ny) * ez)]) return true;
  return false;
}

// visit every node within +-2 of `node` (in each direction) that shares a fluid element
template <typename F>
static void for_neighbors(const MeshHost& M, int64_t node, F f) {
  // mark the nodes of the fluid elements that hold `node` in its 5 x 5 x 5 window, then visit
  // the marks in window order (= increasing node index)
  int i, j, k, ei[2], ej[2], ek[2];
  M.coords(node, i, j, k);
  const int ni = elem_range(i, M.nx, ei), nj = elem_range(j, M.ny, ej), nk = elem_range(k, M.nz, ek);
  bool mark[125] = {};
  bool any = false;
  for (int c = 0; c < nk; ++c)
    for (int b = 0; b < nj; ++b)
      for (int a = 0; a < ni; ++a) {
        if (!M.mask[ei[a] + int64_t(M.nx) * (ej[b] + int64_t(M.ny) * ek[c])]) continue;
        any = true;
        const int x0 = 2 * ei[a] - i + 2, y0 = 2 * ej[b] - j + 2, z0 = 2 * ek[c] - k + 2;  // element corner in the window
        for (int z = 0; z < 3; ++z)
          for (int y = 0; y < 3; ++y)
            for (int x = 0; x < 3; ++x) mark[(x0 + x) + 5 * ((y0 + y) + 5 * (z0 + z))] = true;
      }
  if (!any) return;
  for (int dz = 0; dz < 5; ++dz)
    for (int dy = 0; dy < 5; ++dy)
      for (int dx = 0; dx < 5; ++dx)
        if (mark[dx + 5 * (dy + 5 * dz)])
          f(int64_t(i + dx - 2) + int64_t(M.NX) * (int64_t(j + dy - 2) + int64_t(M.NY) * (k + dz - 2)));
}

// ------------------------------------------------------------------ mesh and patterns
// Sliced layout of the velocity rows for the SpMV: on GB300 an FP64 warp instruction costs
// the same with 1 or 32 active lanes, so each lane takes one whole row and the rows of a warp
// are made to have (nearly) the same number of blocks.
static void build_sell(MeshHost& M) {
  const int64_t nv = M.nv;
  const int64_t W = 1024;
  std::vector<int32_t> order(nv);
  for (int64_t r = 0; r < nv; ++r) order[r] = int32_t(r);
  auto alen = [&](int32_t r) { return M.a_ptr[r + 1] - M.a_ptr[r]; };
  auto blen = [&](int32_t r) { return M.bt_ptr[r + 1] - M.bt_ptr[r]; };
  parallel_tasks((nv + W - 1) / W, [&](int64_t q) {
    const int64_t w0 = q * W;
    auto b = order.begin() + w0, e = order.begin() + std::min(nv, w0 + W);
    std::sort(b, e, [&](int32_t x, int32_t y) {
      if (alen(x) != alen(y)) return alen(x) > alen(y);
      if (blen(x) != blen(y)) return blen(x) > blen(y);
      return x < y;
    });
  });
  const int64_t ns = (nv + 31) / 32;
  M.sell_row.assign(ns * 32, -1);
  M.sell_aoff.assign(ns + 1, 0);
  M.sell_boff.assign(ns + 1, 0);
  for (int64_t sl = 0; sl < ns; ++sl) {
    int la = 0, lb = 0;
    for (int l = 0; l < 32 && sl * 32 + l < nv; ++l) {
      const int32_t r = order[sl * 32 + l];
      M.sell_row[sl * 32 + l] = r;
      la = std::max(la, alen(r));
      lb = std::max(lb, blen(r));
    }
    M.sell_aoff[sl + 1] = M.sell_aoff[sl] + int64_t(la) * 32;
    M.sell_boff[sl + 1] = M.sell_boff[sl] + int64_t(lb) * 32;
  }
  M.sell_acol.assign(M.sell_aoff[ns], 0);
  M.sell_asrc.assign(M.sell_aoff[ns], -1);
  M.sell_bcol.assign(M.sell_boff[ns], 0);
  M.sell_bsrc.assign(M.sell_boff[ns], -1);
  parallel_for(ns, [&](int64_t sl) {
    for (int l = 0; l < 32; ++l) {
      const int32_t r = M.sell_row[sl * 32 + l];
      if (r < 0) continue;
      for (int j = 0; j < alen(r); ++j) {
        const int64_t slot = M.sell_aoff[sl] + int64_t(j) * 32 + l;
        M.sell_acol[slot] = M.a_col[M.a_ptr[r] + j];
        M.sell_asrc[slot] = M.a_ptr[r] + j;
      }
      for (int j = 0; j < blen(r); ++j) {
        const int64_t slot = M.sell_boff[sl] + int64_t(j) * 32 + l;
        M.sell_bcol[slot] = M.bt_col[M.bt_ptr[r] + j];
        M.sell_bsrc[slot] = M.bt_ptr[r] + j;
      }
    }
  });
}

// The 27 Q2 nodes of element e, in local order a = x + 3 y + 9 z.
static void element_nodes(const MeshHost& M, int64_t e, int64_t out[27]) {
  const int ex = int(e % M.nx), ey = int((e / M.nx) % M.ny), ez = int(e / (int64_t(M.nx) * M.ny));
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a)
        out[a + 3 * b + 9 * c] = (2 * ex + a) + int64_t(M.NX) * ((2 * ey + b) + int64_t(M.NY) * (2 * ez + c));
}

// P1-disc patterns (Section 2 element pair): pressure row 4 f + k couples to the free velocity
// nodes of fluid element f (and, for the lifting, to its Dirichlet nodes with a nonzero datum);
// velocity node I couples to the four pressure dofs of every fluid element holding it.  All
// lists ascending (node order equals velocity-index order; fluid rank order equals element order).
static void build_p1disc_patterns(MeshHost& M) {
  const int64_t nf = int64_t(M.fluid.size());
  std::vector<int32_t> rv(nf * 27), rn(nf * 27), dv(nf * 27), dn(nf * 27);
  parallel_for(nf, [&](int64_t f) {
    int64_t nd[27];
    element_nodes(M, M.fluid[f], nd);
    std::sort(nd, nd + 27);
    int a = 0, b = 0;
    for (int q = 0; q < 27; ++q) {
      const int64_t v = nd[q];
      if (M.vidx[v] >= 0) rv[f * 27 + a++] = M.vidx[v];
      const uint8_t t = M.tags[v];
      const bool nz = M.g[3 * v] != 0.0 || M.g[3 * v + 1] != 0.0 || M.g[3 * v + 2] != 0.0;
      if ((t == GDSW_TAG_WALL || t == GDSW_TAG_INFLOW) && nz) dv[f * 27 + b++] = int32_t(v);
    }
    rn[f] = a;
    dn[f] = b;
  });
  M.b_ptr.assign(4 * nf + 1, 0);
  M.bd_ptr.assign(4 * nf + 1, 0);
  for (int64_t f = 0; f < nf; ++f)
    for (int k = 0; k < 4; ++k) {
      M.b_ptr[4 * f + k + 1] = M.b_ptr[4 * f + k] + rn[f];
      M.bd_ptr[4 * f + k + 1] = M.bd_ptr[4 * f + k] + dn[f];
    }
  M.b_col.resize(M.b_ptr[4 * nf]);
  M.bd_col.resize(M.bd_ptr[4 * nf]);
  parallel_for(nf, [&](int64_t f) {
    for (int k = 0; k < 4; ++k) {
      std::copy(rv.begin() + f * 27, rv.begin() + f * 27 + rn[f], M.b_col.begin() + M.b_ptr[4 * f + k]);
      std::copy(dv.begin() + f * 27, dv.begin() + f * 27 + dn[f], M.bd_col.begin() + M.bd_ptr[4 * f + k]);
    }
  });
  // velocity rows: the fluid elements holding the node, ascending
  M.bt_ptr.assign(M.nv + 1, 0);
  std::vector<int32_t> ecount(M.nv, 0);
  parallel_for(M.nv, [&](int64_t I) {
    int i, j, k, ei[2], ej[2], ek[2];
    M.coords(M.vnode[I], i, j, k);
    const int ni = elem_range(i, M.nx, ei), nj = elem_range(j, M.ny, ej), nk = elem_range(k, M.nz, ek);
    int c = 0;
    for (int z = 0; z < nk; ++z)
      for (int y = 0; y < nj; ++y)
        for (int x = 0; x < ni; ++x) c += M.felem[ei[x] + int64_t(M.nx) * (ej[y] + int64_t(M.ny) * ek[z])] >= 0;
    ecount[I] = c;
  });
  for (int64_t I = 0; I < M.nv; ++I) M.bt_ptr[I + 1] = M.bt_ptr[I] + 4 * ecount[I];
  M.bt_col.resize(M.bt_ptr[M.nv]);
  parallel_for(M.nv, [&](int64_t I) {
    int i, j, k, ei[2], ej[2], ek[2];
    M.coords(M.vnode[I], i, j, k);
    const int ni = elem_range(i, M.nx, ei), nj = elem_range(j, M.ny, ej), nk = elem_range(k, M.nz, ek);
    int32_t fl[8];
    int c = 0;
    for (int z = 0; z < nk; ++z)
      for (int y = 0; y < nj; ++y)
        for (int x = 0; x < ni; ++x) {
          const int32_t f = M.felem[ei[x] + int64_t(M.nx) * (ej[y] + int64_t(M.ny) * ek[z])];
          if (f >= 0) fl[c++] = f;
        }
    std::sort(fl, fl + c);
    int32_t* out = M.bt_col.data() + M.bt_ptr[I];
    for (int q = 0; q < c; ++q)
      for (int kk = 0; kk < 4; ++kk) out[4 * q + kk] = 4 * fl[q] + kk;
  });
}

void build_mesh(MeshHost& M, const gdsw_mesh* m) {
  M.nx = m->nx; M.ny = m->ny; M.nz = m->nz;
  M.h = m->h;
  for (int d = 0; d < 3; ++d) M.origin[d] = m->origin[d];
  M.NX = 2 * M.nx + 1; M.NY = 2 * M.ny + 1; M.NZ = 2 * M.nz + 1;
  M.nnodes = int64_t(M.NX) * M.NY * M.NZ;
  int64_t ne = int64_t(M.nx) * M.ny * M.nz;
  M.mask.assign(m->mask, m->mask + ne);
  M.tags.assign(m->tags, m->tags + M.nnodes);
  M.g.assign(m->g, m->g + 3 * M.nnodes);
  M.felem.assign(ne, -1);
  M.fluid.clear();
  for (int64_t e = 0; e < ne; ++e)
    if (M.mask[e]) {
      M.felem[e] = int32_t(M.fluid.size());
      M.fluid.push_back(int32_t(e));
    }
  GDSW_CHECK(!M.fluid.empty(), GDSW_ERR_INVALID_ARG, "mesh has no fluid element");
  M.active.assign(M.nnodes, 0);
  for (int32_t e : M.fluid) {
    int ex = e % M.nx, ey = (e / M.nx) % M.ny, ez = e / (M.nx * M.ny);
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a)
          M.active[(2 * ex + a) + int64_t(M.NX) * ((2 * ey + b) + int64_t(M.NY) * (2 * ez + c))] = 1;
  }
  GDSW_CHECK(m->pressure == GDSW_PRESSURE_Q1 || m->pressure == GDSW_PRESSURE_P1DISC, GDSW_ERR_INVALID_ARG,
             "unknown pressure element");
  M.pdisc = m->pressure == GDSW_PRESSURE_P1DISC;
  M.vidx.assign(M.nnodes, -1);
  M.pidx.assign(M.nnodes, -1);
  M.vnode.clear();
  M.pnode.clear();
  for (int64_t v = 0; v < M.nnodes; ++v) {
    if (!M.active[v]) continue;
    uint8_t t = M.tags[v];
    if (t != GDSW_TAG_WALL && t != GDSW_TAG_INFLOW) {
      M.vidx[v] = int32_t(M.vnode.size());
      M.vnode.push_back(int32_t(v));
    }
    int i, j, k;
    M.coords(v, i, j, k);
    if (!M.pdisc && i % 2 == 0 && j % 2 == 0 && k % 2 == 0) {
      M.pidx[v] = int32_t(M.pnode.size());
      M.pnode.push_back(int32_t(v));
    }
  }
  M.nv = int64_t(M.vnode.size());
  M.np = M.pdisc ? 4 * int64_t(M.fluid.size()) : int64_t(M.pnode.size());
  M.nu = 3 * M.nv;
  M.n = M.nu + M.np;
  GDSW_CHECK(M.n < (int64_t(1) << 31), GDSW_ERR_INVALID_ARG, "problem too large for int32 dof indices");

  // neighbour lists per row node, all three kinds from one scan of the neighbours: free
  // velocity nodes, pressure nodes, Dirichlet nodes with a nonzero datum (the only ones the
  // lifting needs); lists in increasing index
  auto build = [&](const std::vector<int32_t>& rows, std::vector<int32_t>* ptr[3], std::vector<int32_t>* col[3]) {
    const int64_t nr = int64_t(rows.size());
    std::vector<std::vector<int32_t>> tmp[3];
    for (int k = 0; k < 3; ++k)
      if (ptr[k]) tmp[k].resize(nr);
    parallel_for(nr, [&](int64_t r) {
      for_neighbors(M, rows[r], [&](int64_t w) {
        if (ptr[0] && M.vidx[w] >= 0) tmp[0][r].push_back(M.vidx[w]);
        if (ptr[1] && M.pidx[w] >= 0) tmp[1][r].push_back(M.pidx[w]);
        if (ptr[2]) {
          const uint8_t t = M.tags[w];
          const bool nz = M.g[3 * w] != 0.0 || M.g[3 * w + 1] != 0.0 || M.g[3 * w + 2] != 0.0;
          if ((t == GDSW_TAG_WALL || t == GDSW_TAG_INFLOW) && nz) tmp[2][r].push_back(int32_t(w));
        }
      });
      for (int k = 0; k < 3; ++k)
        if (ptr[k]) std::sort(tmp[k][r].begin(), tmp[k][r].end());
    });
    for (int k = 0; k < 3; ++k) {
      if (!ptr[k]) continue;
      ptr[k]->assign(nr + 1, 0);
      for (int64_t r = 0; r < nr; ++r) (*ptr[k])[r + 1] = (*ptr[k])[r] + int32_t(tmp[k][r].size());
      col[k]->resize((*ptr[k])[nr]);
      parallel_for(nr, [&](int64_t r) {
        std::copy(tmp[k][r].begin(), tmp[k][r].end(), col[k]->begin() + (*ptr[k])[r]);
      });
    }
  };
  {
    std::vector<int32_t>* vp[3] = {&M.a_ptr, &M.bt_ptr, &M.ad_ptr};
    std::vector<int32_t>* vc[3] = {&M.a_col, &M.bt_col, &M.ad_col};
    build(M.vnode, vp, vc);
    std::vector<int32_t>* pp[3] = {&M.b_ptr, nullptr, &M.bd_ptr};
    std::vector<int32_t>* pc[3] = {&M.b_col, nullptr, &M.bd_col};
    build(M.pnode, pp, pc);
  }
  if (M.pdisc) {
    // an element's pressure dofs travel with its centre node in the local orderings
    for (int32_t e : M.fluid) {
      int64_t nd[27];
      element_nodes(M, e, nd);
      GDSW_CHECK(M.vidx[nd[13]] >= 0, GDSW_ERR_INVALID_ARG, "P1-disc: an element centre node has no free velocity");
    }
    build_p1disc_patterns(M);
  }
  // symmetric velocity pattern: diagonal block of each row and the transpose of each block
  M.a_diag.assign(M.nv, -1);
  M.a_tpos.resize(M.a_col.size());
  std::atomic<int> asym(0);
  parallel_for(M.nv, [&](int64_t I) {
    for (int32_t blk = M.a_ptr[I]; blk < M.a_ptr[I + 1]; ++blk) {
      int32_t J = M.a_col[blk];
      if (J == I) M.a_diag[I] = blk;
      auto r0 = M.a_col.begin() + M.a_ptr[J], r1 = M.a_col.begin() + M.a_ptr[J + 1];
      auto it = std::lower_bound(r0, r1, int32_t(I));
      if (it == r1 || *it != int32_t(I)) {
        asym = 1;
        continue;
      }
      M.a_tpos[blk] = int32_t(it - M.a_col.begin());
    }
  });
  GDSW_CHECK(asym == 0, GDSW_ERR_INVALID_ARG, "asymmetric velocity pattern");
  for (int64_t I = 0; I < M.nv; ++I) GDSW_CHECK(M.a_diag[I] >= 0, GDSW_ERR_INVALID_ARG, "missing diagonal block");
  // assembly units: for each upper block, the fluid elements holding both nodes
  GDSW_CHECK(int64_t(M.fluid.size()) < (int64_t(1) << 22), GDSW_ERR_INVALID_ARG,
             "too many fluid elements for the packed assembly units");
  const int64_t nnzb = int64_t(M.a_col.size());
  std::vector<int32_t> ucount(nnzb, 0);
  auto units_of = [&](int64_t I, int32_t blk, uint32_t* out) {
    int ii[3], jj[3];
    M.coords(M.vnode[I], ii[0], ii[1], ii[2]);
    M.coords(M.vnode[M.a_col[blk]], jj[0], jj[1], jj[2]);
    const int nn[3] = {M.nx, M.ny, M.nz};
    int e0[3], e1[3];
    for (int d = 0; d < 3; ++d) {
      const int lo = std::max(ii[d], jj[d]), hi = std::min(ii[d], jj[d]);
      e0[d] = lo < 2 ? 0 : (lo - 1) / 2;
      e1[d] = std::min(nn[d] - 1, hi / 2);
    }
    int cnt = 0;
    for (int ez = e0[2]; ez <= e1[2]; ++ez)
      for (int ey = e0[1]; ey <= e1[1]; ++ey)
        for (int ex = e0[0]; ex <= e1[0]; ++ex) {
          const int64_t e = ex + int64_t(M.nx) * (ey + int64_t(M.ny) * ez);
          if (!M.mask[e]) continue;
          if (out) {
            const uint32_t a = uint32_t((ii[0] - 2 * ex) + 3 * (ii[1] - 2 * ey) + 9 * (ii[2] - 2 * ez));
            const uint32_t b = uint32_t((jj[0] - 2 * ex) + 3 * (jj[1] - 2 * ey) + 9 * (jj[2] - 2 * ez));
            out[cnt] = (uint32_t(M.felem[e]) << 10) | (a << 5) | b;
          }
          ++cnt;
        }
    return cnt;
  };
  parallel_for(M.nv, [&](int64_t I) {
    for (int32_t blk = M.a_diag[I]; blk < M.a_ptr[I + 1]; ++blk) ucount[blk] = units_of(I, blk, nullptr);
  });
  M.asm_uoff.assign(nnzb + 1, 0);
  for (int64_t q = 0; q < nnzb; ++q) M.asm_uoff[q + 1] = M.asm_uoff[q] + ucount[q];
  GDSW_CHECK(int64_t(M.asm_uoff[nnzb]) < (int64_t(1) << 31), GDSW_ERR_INVALID_ARG, "too many assembly units");
  M.asm_unit.resize(M.asm_uoff[nnzb]);
  parallel_for(M.nv, [&](int64_t I) {
    for (int32_t blk = M.a_diag[I]; blk < M.a_ptr[I + 1]; ++blk) units_of(I, blk, M.asm_unit.data() + M.asm_uoff[blk]);
  });
  M.asm_cta.assign(1, 0);
  for (int64_t q = 0; q < nnzb; ++q)
    if (M.asm_uoff[q + 1] - M.asm_uoff[M.asm_cta.back()] > 256) M.asm_cta.push_back(int32_t(q));
  M.asm_cta.push_back(int32_t(nnzb));
  // BT entry (I, P) has the value of B entry (P, I)
  M.bt2b.resize(M.bt_col.size());
  std::atomic<int> basym(0);
  parallel_for(M.nv, [&](int64_t I) {
    for (int32_t e = M.bt_ptr[I]; e < M.bt_ptr[I + 1]; ++e) {
      int32_t P = M.bt_col[e];
      auto b0 = M.b_col.begin() + M.b_ptr[P], b1 = M.b_col.begin() + M.b_ptr[P + 1];
      auto it = std::lower_bound(b0, b1, int32_t(I));
      if (it == b1 || *it != int32_t(I)) {
        basym = 1;
        continue;
      }
      M.bt2b[e] = int32_t(it - M.b_col.begin());
    }
  });
  GDSW_CHECK(basym == 0, GDSW_ERR_INVALID_ARG, "asymmetric B pattern");
  build_sell(M);
}

// ------------------------------------------------------------------ slab layout
void SlabSet::layout() {
  nsub = int(K.size());
  voff.assign(nsub + 1, 0);
  soff.assign(nsub, {});
  fS.assign(nsub, {}); fG.assign(nsub, {}); fW.assign(nsub, {});
  ldS.assign(nsub, {}); ldG.assign(nsub, {}); ldW.assign(nsub, {});
  nfac = 0;
  Kmax = 0;
  max_local = 0;
  for (int i = 0; i < nsub; ++i) {
    Kmax = std::max(Kmax, K[i]);
    int64_t off = 0;
    for (int k = 0; k < K[i]; ++k) {
      soff[i].push_back(off);
      off += s[i][k];
    }
    voff[i + 1] = voff[i] + off;
    max_local = std::max(max_local, off);
    for (int k = 0; k < K[i]; ++k) {
      int sk = s[i][k];
      int ld = int(pad8(sk));
      ldS[i].push_back(ld);
      fS[i].push_back(nfac);
      nfac += int64_t(sk) * ld;
      // G_k: m_k x s_{k-1}
      int ldg = k > 0 ? int(pad8(s[i][k - 1])) : 8;
      ldG[i].push_back(ldg);
      fG[i].push_back(nfac);
      if (k > 0) nfac += int64_t(m[i][k]) * ldg;
      // W_k = S_k^{-1} C_k is not stored: the operator is symmetric, so W_k = G_{k+1}^T
      ldW[i].push_back(8);
      fW[i].push_back(-1);
    }
  }
  nvec = voff[nsub];
}

// P1-disc pressure dofs that an element adds to a dof set (they belong to no node).  high:
// the dofs join the slab of the element's last node plane across the slab axis, else the slab
// of its centre.  A set of whole elements (an overlapping subdomain, whose element constants
// are free) needs `high`: a leading block of the block-tridiagonal factorisation then holds an
// element's constant only together with every one of its velocity nodes, so the constant
// pressure on the elements of the leading slabs is never a kernel of the leading block.  The
// linear dofs of an interior set are controlled by the element's centre (bubble) node alone.
struct ElemDofs {
  int64_t e;
  int n;
  int32_t d[4];
  bool high;
};

// Order the free dofs of a node set for a block-tridiagonal factorisation: slabs of
// `t` element layers across the longest axis of the set (t = 0: one slab); inside each
// slab the dofs of nodes coupled to the previous slab come first.  Appends to `S`.
static void slab_order(const MeshHost& M, std::vector<int64_t> nodes, int t, SlabSet& S,
                       const std::vector<ElemDofs>* edofs = nullptr) {
  std::sort(nodes.begin(), nodes.end());
  if (nodes.empty()) {
    S.K.push_back(0);
    S.s.push_back({});
    S.m.push_back({});
    return;
  }
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
  for (int64_t v : nodes) {
    int c[3];
    M.coords(v, c[0], c[1], c[2]);
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], c[d]);
      hi[d] = std::max(hi[d], c[d]);
    }
  }
  int ax = 0;
  for (int d = 1; d < 3; ++d)
    if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
  int c0 = lo[ax] - (lo[ax] % 2);
  // membership lookup over the bounding box
  int bx = hi[0] - lo[0] + 1, by = hi[1] - lo[1] + 1, bz = hi[2] - lo[2] + 1;
  std::vector<int32_t> box(int64_t(bx) * by * bz, -1);
  auto bidx = [&](int i, int j, int k) { return (i - lo[0]) + int64_t(bx) * ((j - lo[1]) + int64_t(by) * (k - lo[2])); };
  std::vector<int> raw(nodes.size());
  for (size_t q = 0; q < nodes.size(); ++q) {
    int c[3];
    M.coords(nodes[q], c[0], c[1], c[2]);
    box[bidx(c[0], c[1], c[2])] = int32_t(q);
    raw[q] = t > 0 ? (c[ax] - c0) / (2 * t) : 0;
  }
  std::vector<int> uniq(raw);
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  std::vector<int> slab(nodes.size());
  for (size_t q = 0; q < nodes.size(); ++q)
    slab[q] = int(std::lower_bound(uniq.begin(), uniq.end(), raw[q]) - uniq.begin());
  int K = int(uniq.size());
  std::vector<uint8_t> back(nodes.size(), 0);
  for (size_t q = 0; q < nodes.size(); ++q) {
    if (slab[q] == 0) continue;
    int c[3];
    M.coords(nodes[q], c[0], c[1], c[2]);
    bool found = false;
    for (int dk = -2; dk <= 2 && !found; ++dk)
      for (int dj = -2; dj <= 2 && !found; ++dj)
        for (int di = -2; di <= 2 && !found; ++di) {
          int i = c[0] + di, j = c[1] + dj, k = c[2] + dk;
          if (i < lo[0] || i > hi[0] || j < lo[1] || j > hi[1] || k < lo[2] || k > hi[2]) continue;
          int32_t w = box[bidx(i, j, k)];
          if (w < 0 || slab[w] != slab[q] - 1) continue;
          if (M.shares_element(nodes[q], nodes[w])) found = true;
        }
    back[q] = found;
  }
  std::vector<std::vector<int32_t>> A(K), B(K);
  for (size_t q = 0; q < nodes.size(); ++q) {
    int64_t v = nodes[q];
    auto& dst = back[q] ? A[slab[q]] : B[slab[q]];
    if (M.vidx[v] >= 0)
      for (int c = 0; c < 3; ++c) dst.push_back(int32_t(3 * M.vidx[v] + c));
    if (M.pidx[v] >= 0) dst.push_back(int32_t(M.nu + M.pidx[v]));
  }
  if (edofs) {
    auto member = [&](int i, int j, int k) -> int32_t {
      if (i < lo[0] || i > hi[0] || j < lo[1] || j > hi[1] || k < lo[2] || k > hi[2]) return -1;
      return box[bidx(i, j, k)];
    };
    auto slab_of_raw = [&](int r) {
      auto it = std::lower_bound(uniq.begin(), uniq.end(), r);
      return (it != uniq.end() && *it == r) ? int(it - uniq.begin()) : -1;
    };
    for (const ElemDofs& x : *edofs) {
      const int ec[3] = {int(x.e % M.nx), int((x.e / M.nx) % M.ny), int(x.e / (int64_t(M.nx) * M.ny))};
      const int centre = 2 * ec[ax] + 1;
      const int rc = t > 0 ? (centre - c0) / (2 * t) : 0;
      int sl = -1;
      if (x.high) sl = slab_of_raw(t > 0 ? (centre + 1 - c0) / (2 * t) : 0);
      if (sl < 0) sl = slab_of_raw(rc);
      GDSW_CHECK(sl >= 0, GDSW_ERR_INVALID_ARG, "element pressure dofs without their element's nodes");
      bool bk = false;
      for (int z = 0; z < 3 && !bk; ++z)
        for (int y = 0; y < 3 && !bk; ++y)
          for (int w = 0; w < 3 && !bk; ++w) {
            const int32_t q = member(2 * ec[0] + w, 2 * ec[1] + y, 2 * ec[2] + z);
            if (q >= 0 && slab[q] == sl - 1) bk = true;
          }
      auto& dst = bk ? A[sl] : B[sl];
      for (int c = 0; c < x.n; ++c) dst.push_back(x.d[c]);
    }
  }
  std::vector<int> s, m;
  for (int k = 0; k < K; ++k) {
    std::sort(A[k].begin(), A[k].end());
    std::sort(B[k].begin(), B[k].end());
    s.push_back(int(A[k].size() + B[k].size()));
    m.push_back(int(A[k].size()));
    S.gdof.insert(S.gdof.end(), A[k].begin(), A[k].end());
    S.gdof.insert(S.gdof.end(), B[k].begin(), B[k].end());
  }
  // drop empty slabs (a slab can be empty of dofs if all its nodes are Dirichlet-only)
  std::vector<int> s2, m2;
  for (int k = 0; k < K; ++k)
    if (s[k] > 0) {
      s2.push_back(s[k]);
      m2.push_back(m[k]);
    } else if (k + 1 < K) {
      m[k + 1] = 0;
    }
  if (!s2.empty()) m2[0] = 0;
  S.K.push_back(int(s2.size()));
  S.s.push_back(s2);
  S.m.push_back(m2);
}

// One dense block holding sorted dofs (coarse levels).
static void dense_order(const std::vector<int32_t>& dofs, SlabSet& S) {
  std::vector<int32_t> d(dofs);
  std::sort(d.begin(), d.end());
  if (d.empty()) {
    S.K.push_back(0);
    S.s.push_back({});
    S.m.push_back({});
    return;
  }
  S.K.push_back(1);
  S.s.push_back({int(d.size())});
  S.m.push_back({0});
  S.gdof.insert(S.gdof.end(), d.begin(), d.end());
}

static void scatter_lists(LevelHost& L, int weighting) {
  const SlabSet& S = L.loc;
  std::vector<int32_t> mult(L.n, 0);
  for (int32_t g : S.gdof) mult[g]++;
  L.sc_ptr.assign(L.n + 1, 0);
  for (int32_t g : S.gdof) L.sc_ptr[g + 1]++;
  for (int g = 0; g < L.n; ++g) L.sc_ptr[g + 1] += L.sc_ptr[g];
  L.sc_pos.resize(S.gdof.size());
  L.sc_w.resize(S.gdof.size());
  std::vector<int32_t> fill(L.sc_ptr.begin(), L.sc_ptr.end() - 1);
  for (int64_t p = 0; p < int64_t(S.gdof.size()); ++p) {
    int32_t g = S.gdof[p];
    L.sc_pos[fill[g]] = int32_t(p);
    L.sc_w[fill[g]] = weighting == GDSW_WEIGHT_POU ? 1.0 / double(mult[g]) : 1.0;
    fill[g]++;
  }
  // sorted overlapping dof lists per part
  L.dof_off.assign(S.nsub + 1, 0);
  L.dof_sorted.clear();
  for (int i = 0; i < S.nsub; ++i) {
    std::vector<int32_t> d(S.gdof.begin() + S.voff[i], S.gdof.begin() + S.voff[i + 1]);
    std::sort(d.begin(), d.end());
    L.dof_sorted.insert(L.dof_sorted.end(), d.begin(), d.end());
    L.dof_off[i + 1] = int64_t(L.dof_sorted.size());
  }
}

// restriction lists and part column lists, shared by every level
static void coarse_lists(CoarseSpace& C, const std::vector<std::vector<int>>& ent_set,
                         const std::vector<std::vector<int>>& ent_cols) {
  // columns of every part: columns of entities whose set contains the part
  std::vector<std::vector<int32_t>> pc(C.nparts);
  for (size_t e = 0; e < ent_set.size(); ++e)
    for (int p : ent_set[e])
      for (int c : ent_cols[e]) pc[p].push_back(c);
  C.coff.assign(C.nparts + 1, 0);
  C.cols.clear();
  for (int p = 0; p < C.nparts; ++p) {
    std::sort(pc[p].begin(), pc[p].end());
    C.cols.insert(C.cols.end(), pc[p].begin(), pc[p].end());
    C.coff[p + 1] = int64_t(C.cols.size());
  }
  // restriction reduce: coarse column k <- parts in increasing order
  std::vector<std::vector<int32_t>> rr(C.n0);
  for (int p = 0; p < C.nparts; ++p)
    for (int64_t q = C.coff[p]; q < C.coff[p + 1]; ++q) rr[C.cols[q]].push_back(int32_t(q));
  C.rr_ptr.assign(C.n0 + 1, 0);
  C.rr_pos.clear();
  for (int k = 0; k < C.n0; ++k) {
    C.rr_pos.insert(C.rr_pos.end(), rr[k].begin(), rr[k].end());
    C.rr_ptr[k + 1] = int32_t(C.rr_pos.size());
  }
  if (C.gval.size() != C.gdofs.size()) C.gval.assign(C.gdofs.size(), 1.0);  // indicator entries
  std::vector<std::vector<std::pair<int32_t, double>>> rg(C.n0);
  for (size_t q = 0; q < C.gdofs.size(); ++q) rg[C.gcol[q]].push_back({C.gdofs[q], C.gval[q]});
  C.rg_ptr.assign(C.n0 + 1, 0);
  C.rg_dof.clear();
  C.rg_val.clear();
  for (int k = 0; k < C.n0; ++k) {
    std::sort(rg[k].begin(), rg[k].end());
    for (auto& e : rg[k]) {
      C.rg_dof.push_back(e.first);
      C.rg_val.push_back(e.second);
    }
    C.rg_ptr[k + 1] = int32_t(C.rg_dof.size());
  }
  // entries grouped by interface dof (gdofs ascending): prolongation, one thread per dof
  C.gu_dof.clear();
  C.gu_ptr.assign(1, 0);
  for (size_t q = 0; q < C.gdofs.size(); ++q) {
    if (q == 0 || C.gdofs[q] != C.gdofs[q - 1]) {
      if (q > 0) C.gu_ptr.push_back(int32_t(q));
      C.gu_dof.push_back(C.gdofs[q]);
    }
  }
  if (!C.gdofs.empty()) C.gu_ptr.push_back(int32_t(C.gdofs.size()));
}

// ------------------------------------------------------------------ level 1
void build_level1(gdsw_ctx* ctx, const gdsw_partition* part, int overlap, int slab_elems, int rotations) {
  MeshHost& M = ctx->mesh;
  LevelHost& L = ctx->lh[0];
  const int64_t ne = int64_t(M.nx) * M.ny * M.nz;
  std::vector<int32_t> ep(ne, -1);
  int N = 0;
  for (int32_t e : M.fluid) {
    int32_t p = part->elem_part[e];
    GDSW_CHECK(p >= 0, GDSW_ERR_INVALID_ARG, "fluid element without subdomain");
    ep[e] = p;
    N = std::max(N, p + 1);
  }
  L.n = int(M.n);
  L.N = N;
  // element bounding boxes per subdomain
  std::vector<std::array<int, 6>> bb(N, {1 << 30, 1 << 30, 1 << 30, -1, -1, -1});
  std::vector<int> cnt(N, 0);
  for (int32_t e : M.fluid) {
    int c[3] = {int(e % M.nx), int((e / M.nx) % M.ny), int(e / (int64_t(M.nx) * M.ny))};
    auto& b = bb[ep[e]];
    for (int d = 0; d < 3; ++d) {
      b[d] = std::min(b[d], c[d]);
      b[3 + d] = std::max(b[3 + d], c[d]);
    }
    cnt[ep[e]]++;
  }
  for (int i = 0; i < N; ++i) GDSW_CHECK(cnt[i] > 0, GDSW_ERR_INVALID_ARG, "empty subdomain id");
  // sharing sets of active nodes
  std::vector<std::array<int32_t, 8>> sh(M.nnodes);
  std::vector<uint8_t> nsh(M.nnodes, 0);
  parallel_for(M.nnodes, [&](int64_t v) {
    if (!M.active[v]) return;
    int i, j, k, ei[2], ej[2], ek[2];
    M.coords(v, i, j, k);
    int ni = elem_range(i, M.nx, ei), nj = elem_range(j, M.ny, ej), nk = elem_range(k, M.nz, ek);
    int32_t tmp[8];
    int c = 0;
    for (int a = 0; a < nk; ++a)
      for (int b = 0; b < nj; ++b)
        for (int d = 0; d < ni; ++d) {
          int64_t e = ei[d] + int64_t(M.nx) * (ej[b] + int64_t(M.ny) * ek[a]);
          if (M.mask[e]) tmp[c++] = ep[e];
        }
    std::sort(tmp, tmp + c);
    int u = int(std::unique(tmp, tmp + c) - tmp);
    for (int q = 0; q < u; ++q) sh[v][q] = tmp[q];
    nsh[v] = uint8_t(u);
  });
  auto has_free = [&](int64_t v) { return M.vidx[v] >= 0 || M.pidx[v] >= 0; };

  // ---- overlapping subdomains (Section 2.1: k layers of elements) ----
  std::vector<std::vector<int64_t>> onodes(N);
  std::vector<std::vector<int32_t>> oelems(N);   // P1-disc: fluid ranks whose pressure is kept
  parallel_tasks(N, [&](int64_t i) {
    int lo[3], hi[3], nn[3] = {M.nx, M.ny, M.nz};
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::max(0, bb[i][d] - overlap);
      hi[d] = std::min(nn[d] - 1, bb[i][3 + d] + overlap);
    }
    int E[3] = {hi[0] - lo[0] + 1, hi[1] - lo[1] + 1, hi[2] - lo[2] + 1};
    int V[3] = {2 * E[0] + 1, 2 * E[1] + 1, 2 * E[2] + 1};
    std::vector<uint8_t> em(int64_t(E[0]) * E[1] * E[2], 0), nm(int64_t(V[0]) * V[1] * V[2], 0);
    auto gel = [&](int a, int b, int c) { return (lo[0] + a) + int64_t(M.nx) * ((lo[1] + b) + int64_t(M.ny) * (lo[2] + c)); };
    auto lel = [&](int a, int b, int c) { return a + int64_t(E[0]) * (b + int64_t(E[1]) * c); };
    auto lnd = [&](int a, int b, int c) { return a + int64_t(V[0]) * (b + int64_t(V[1]) * c); };
    for (int c = 0; c < E[2]; ++c)
      for (int b = 0; b < E[1]; ++b)
        for (int a = 0; a < E[0]; ++a) em[lel(a, b, c)] = (ep[gel(a, b, c)] == i);
    for (int it = 0; it < overlap; ++it) {
      std::fill(nm.begin(), nm.end(), 0);
      for (int c = 0; c < E[2]; ++c)
        for (int b = 0; b < E[1]; ++b)
          for (int a = 0; a < E[0]; ++a)
            if (em[lel(a, b, c)])
              for (int z = 0; z < 3; ++z)
                for (int y = 0; y < 3; ++y)
                  for (int x = 0; x < 3; ++x) nm[lnd(2 * a + x, 2 * b + y, 2 * c + z)] = 1;
      for (int c = 0; c < E[2]; ++c)
        for (int b = 0; b < E[1]; ++b)
          for (int a = 0; a < E[0]; ++a) {
            if (!M.mask[gel(a, b, c)]) continue;
            bool any = false;
            for (int z = 0; z < 3 && !any; ++z)
              for (int y = 0; y < 3 && !any; ++y)
                for (int x = 0; x < 3 && !any; ++x) any = nm[lnd(2 * a + x, 2 * b + y, 2 * c + z)];
            if (any) em[lel(a, b, c)] = 1;
          }
    }
    // nodes whose every fluid element lies in the overlapping subdomain (kn: also the nodes
    // without a free dof, for the P1-disc rule on whole elements)
    std::vector<uint8_t> kn(M.pdisc ? nm.size() : 0, 0);
    for (int c = 0; c < V[2]; ++c)
      for (int b = 0; b < V[1]; ++b)
        for (int a = 0; a < V[0]; ++a) {
          int gi = 2 * lo[0] + a, gj = 2 * lo[1] + b, gk = 2 * lo[2] + c;
          int64_t v = gi + int64_t(M.NX) * (gj + int64_t(M.NY) * gk);
          if (!M.active[v] || (!M.pdisc && !has_free(v))) continue;
          int ei[2], ej[2], ek[2];
          int ni = elem_range(gi, M.nx, ei), nj = elem_range(gj, M.ny, ej), nk = elem_range(gk, M.nz, ek);
          bool all = true;
          for (int z = 0; z < nk && all; ++z)
            for (int y = 0; y < nj && all; ++y)
              for (int x = 0; x < ni && all; ++x) {
                int64_t e = ei[x] + int64_t(M.nx) * (ej[y] + int64_t(M.ny) * ek[z]);
                if (!M.mask[e]) continue;
                int la = ei[x] - lo[0], lb = ej[y] - lo[1], lc = ek[z] - lo[2];
                if (la < 0 || lb < 0 || lc < 0 || la >= E[0] || lb >= E[1] || lc >= E[2] || !em[lel(la, lb, lc)])
                  all = false;
              }
          if (all && M.pdisc) kn[lnd(a, b, c)] = 1;
          if (all && has_free(v)) onodes[i].push_back(v);
        }
    // P1-disc: the pressure dofs of the elements of Omega_i' none of whose nodes lies on its
    // artificial rim (with Dirichlet velocity there the constant pressure on all of Omega_i'
    // would be a kernel of A_i)
    if (M.pdisc)
      for (int c = 0; c < E[2]; ++c)
        for (int b = 0; b < E[1]; ++b)
          for (int a = 0; a < E[0]; ++a) {
            const int64_t e = gel(a, b, c);
            if (!em[lel(a, b, c)] || !M.mask[e]) continue;
            bool all = true;
            for (int z = 0; z < 3 && all; ++z)
              for (int y = 0; y < 3 && all; ++y)
                for (int x = 0; x < 3 && all; ++x) all = kn[lnd(2 * a + x, 2 * b + y, 2 * c + z)] != 0;
            if (all) oelems[i].push_back(M.felem[e]);
          }
  });
  {
    std::vector<SlabSet> parts(N);
    parallel_tasks(N, [&](int64_t i) {
      std::vector<ElemDofs> ed;
      for (int32_t f : oelems[i]) {
        ElemDofs x{M.fluid[f], 4, {}, true};
        for (int k = 0; k < 4; ++k) x.d[k] = int32_t(M.nu + 4 * int64_t(f) + k);
        ed.push_back(x);
      }
      slab_order(M, onodes[i], slab_elems, parts[i], M.pdisc ? &ed : nullptr);
    });
    SlabSet& S = L.loc;
    S = SlabSet();
    for (int i = 0; i < N; ++i) {
      S.K.push_back(parts[i].K[0]);
      S.s.push_back(parts[i].s[0]);
      S.m.push_back(parts[i].m[0]);
      S.gdof.insert(S.gdof.end(), parts[i].gdof.begin(), parts[i].gdof.end());
    }
    S.layout();
  }
  scatter_lists(L, ctx->opt.weighting);

  // ---- interface entities (Section 2.1) ----
  std::map<std::vector<int32_t>, int> gid;
  std::vector<int32_t> grp(M.nnodes, -1);
  std::vector<std::vector<int32_t>> gset;
  for (int64_t v = 0; v < M.nnodes; ++v) {
    if (!M.active[v] || nsh[v] < 2 || !has_free(v)) continue;
    std::vector<int32_t> key(sh[v].begin(), sh[v].begin() + nsh[v]);
    auto it = gid.find(key);
    if (it == gid.end()) {
      it = gid.emplace(key, int(gset.size())).first;
      gset.push_back(key);
    }
    grp[v] = it->second;
  }
  struct Ent { std::vector<int32_t> set; std::vector<int64_t> nodes; };
  std::vector<Ent> ents;
  {
    std::vector<uint8_t> seen(M.nnodes, 0);
    for (int64_t v = 0; v < M.nnodes; ++v) {
      if (grp[v] < 0 || seen[v]) continue;
      Ent E;
      E.set = gset[grp[v]];
      std::vector<int64_t> stack{v};
      seen[v] = 1;
      while (!stack.empty()) {
        int64_t a = stack.back();
        stack.pop_back();
        E.nodes.push_back(a);
        for_neighbors(M, a, [&](int64_t w) {
          if (!seen[w] && grp[w] == grp[a]) {
            seen[w] = 1;
            stack.push_back(w);
          }
        });
      }
      std::sort(E.nodes.begin(), E.nodes.end());
      ents.push_back(std::move(E));
    }
    std::sort(ents.begin(), ents.end(), [](const Ent& a, const Ent& b) {
      if (a.set != b.set) return a.set < b.set;
      return a.nodes[0] < b.nodes[0];
    });
  }
  CoarseSpace& C = L.cs;
  C.n = L.n;
  C.nparts = N;
  C.n_entities = int(ents.size());
  std::vector<std::vector<int>> ent_cols(ents.size());
  int n0 = 0;
  std::vector<std::array<int, 7>> ecol(ents.size());
  // rotations: e_a x (x - x_c) about the centroid x_c of the entity's free velocity nodes, kept
  // when it does not vanish on the entity (the one about a straight edge's own line does)
  std::vector<std::array<double, 3>> centroid(ents.size(), {0.0, 0.0, 0.0});
  auto node_xyz = [&](int64_t v, double x[3]) {
    int i, j, k;
    M.coords(v, i, j, k);
    x[0] = M.origin[0] + 0.5 * M.h * i;
    x[1] = M.origin[1] + 0.5 * M.h * j;
    x[2] = M.origin[2] + 0.5 * M.h * k;
  };
  auto rot_value = [&](size_t e, int64_t v, int a, int comp) {  // (e_a x (x - x_c))_comp
    double x[3];
    node_xyz(v, x);
    double d[3] = {x[0] - centroid[e][0], x[1] - centroid[e][1], x[2] - centroid[e][2]};
    double ea[3] = {0, 0, 0};
    ea[a] = 1.0;
    double cr[3] = {ea[1] * d[2] - ea[2] * d[1], ea[2] * d[0] - ea[0] * d[2], ea[0] * d[1] - ea[1] * d[0]};
    return cr[comp];
  };
  C.cn_set.clear(); C.cn_dofs.clear(); C.cn_modes.clear();
  for (size_t e = 0; e < ents.size(); ++e) {
    bool hv = false, hp = false;
    int nvel = 0;
    for (int64_t v : ents[e].nodes) {
      hv |= M.vidx[v] >= 0;
      hp |= M.pidx[v] >= 0;
      if (M.vidx[v] >= 0) {
        double x[3];
        node_xyz(v, x);
        for (int d = 0; d < 3; ++d) centroid[e][d] += x[d];
        ++nvel;
      }
    }
    if (nvel > 0)
      for (int d = 0; d < 3; ++d) centroid[e][d] /= nvel;
    bool keep_rot[3] = {false, false, false};
    if (rotations && nvel >= 2)
      for (int a = 0; a < 3; ++a) {
        double nrm = 0.0;
        for (int64_t v : ents[e].nodes)
          if (M.vidx[v] >= 0)
            for (int comp = 0; comp < 3; ++comp) nrm += rot_value(e, v, a, comp) * rot_value(e, v, a, comp);
        keep_rot[a] = std::sqrt(nrm) > 1e-8 * M.h;
      }
    std::vector<int> dofs, modes;
    for (int md = 0; md < 7; ++md) {
      bool present = md < 3 ? hv : (md == 3 ? hp : keep_rot[md - 4]);
      ecol[e][md] = present ? n0 : -1;
      if (present) {
        dofs.push_back(n0);
        modes.push_back(md);
        ent_cols[e].push_back(n0);
        n0++;
      }
    }
    C.cn_set.push_back(std::vector<int>(ents[e].set.begin(), ents[e].set.end()));
    C.cn_dofs.push_back(dofs);
    C.cn_modes.push_back(modes);
  }
  // P1-disc: no pressure dof lies on the interface, so the pressure null space enters as one
  // column per subdomain, the constant pressure on the subdomain's own elements (prescribed
  // through the element constants, which join Gamma); none with a single subdomain
  const int n_ent_cols = n0;
  const bool pcols = M.pdisc && N >= 2;
  if (pcols)
    for (int i = 0; i < N; ++i) {
      C.cn_set.push_back({i});
      C.cn_dofs.push_back({n0});
      C.cn_modes.push_back({3});
      ++n0;
    }
  C.n0 = n0;
  C.gdofs.clear();
  C.gcol.clear();
  {
    struct GE { int32_t dof, col; double val; };
    std::vector<GE> gl;
    for (size_t e = 0; e < ents.size(); ++e)
      for (int64_t v : ents[e].nodes) {
        if (M.vidx[v] >= 0)
          for (int c = 0; c < 3; ++c) {
            gl.push_back({int32_t(3 * M.vidx[v] + c), ecol[e][c], 1.0});
            for (int a = 0; a < 3; ++a)
              if (ecol[e][4 + a] >= 0) gl.push_back({int32_t(3 * M.vidx[v] + c), ecol[e][4 + a], rot_value(e, v, a, c)});
          }
        if (M.pidx[v] >= 0) gl.push_back({int32_t(M.nu + M.pidx[v]), ecol[e][3], 1.0});
      }
    if (pcols)
      for (int64_t f = 0; f < int64_t(M.fluid.size()); ++f)
        gl.push_back({int32_t(M.nu + 4 * f), int32_t(n_ent_cols + ep[M.fluid[f]]), 1.0});
    std::sort(gl.begin(), gl.end(), [](const GE& a, const GE& b) { return a.dof != b.dof ? a.dof < b.dof : a.col < b.col; });
    C.gval.clear();
    for (auto& q : gl) {
      C.gdofs.push_back(q.dof);
      C.gcol.push_back(q.col);
      C.gval.push_back(q.val);
    }
  }
  // interiors: nodes whose sharing set is {i}
  std::vector<std::vector<int64_t>> inodes(N);
  for (int64_t v = 0; v < M.nnodes; ++v)
    if (M.active[v] && nsh[v] == 1 && has_free(v)) inodes[sh[v][0]].push_back(v);
  {
    std::vector<SlabSet> parts(N);
    // P1-disc: the pressure dofs of each subdomain's own elements that are not in Gamma (the
    // linear ones; all four with a single subdomain)
    std::vector<std::vector<ElemDofs>> ied(N);
    if (M.pdisc)
      for (int64_t f = 0; f < int64_t(M.fluid.size()); ++f) {
        ElemDofs x{M.fluid[f], 0, {}, false};
        for (int k = pcols ? 1 : 0; k < 4; ++k) x.d[x.n++] = int32_t(M.nu + 4 * f + k);
        ied[ep[M.fluid[f]]].push_back(x);
      }
    parallel_tasks(N, [&](int64_t i) { slab_order(M, inodes[i], slab_elems, parts[i], M.pdisc ? &ied[i] : nullptr); });
    SlabSet& S = L.inter;
    S = SlabSet();
    for (int i = 0; i < N; ++i) {
      S.K.push_back(parts[i].K[0]);
      S.s.push_back(parts[i].s[0]);
      S.m.push_back(parts[i].m[0]);
      S.gdof.insert(S.gdof.end(), parts[i].gdof.begin(), parts[i].gdof.end());
    }
    S.layout();
    C.idofs = S.gdof;
    C.ioff = S.voff;
  }
  std::vector<std::vector<int>> eset(C.cn_set.size());
  for (size_t e = 0; e < C.cn_set.size(); ++e) eset[e] = C.cn_set[e];
  ent_cols.resize(C.cn_set.size());
  for (size_t e = ents.size(); e < C.cn_set.size(); ++e) ent_cols[e] = C.cn_dofs[e];
  coarse_lists(C, eset, ent_cols);
}

// ------------------------------------------------------------------ coarse levels
void build_coarse_level(gdsw_ctx* ctx, int l, const int32_t* group, int group_len) {
  CoarseSpace& P = ctx->lh[l - 1].cs;     // coarse space of the finer level
  LevelHost& L = ctx->lh[l];
  const int nn = int(P.cn_set.size());
  GDSW_CHECK(group_len == P.nparts, GDSW_ERR_INVALID_ARG, "grouping array has the wrong length");
  int N = 0;
  for (int p = 0; p < group_len; ++p) {
    GDSW_CHECK(group[p] >= 0, GDSW_ERR_INVALID_ARG, "negative group id");
    N = std::max(N, group[p] + 1);
  }
  L.n = P.n0;
  L.N = N;
  std::vector<std::vector<int>> R(nn);
  for (int v = 0; v < nn; ++v) {
    for (int p : P.cn_set[v]) R[v].push_back(group[p]);
    std::sort(R[v].begin(), R[v].end());
    R[v].erase(std::unique(R[v].begin(), R[v].end()), R[v].end());
  }
  // coupling: sharing sets intersect
  std::vector<std::vector<int>> byp(P.nparts);
  for (int v = 0; v < nn; ++v)
    for (int p : P.cn_set[v]) byp[p].push_back(v);
  auto neighbors = [&](int v, std::vector<int>& out) {
    out.clear();
    for (int p : P.cn_set[v]) out.insert(out.end(), byp[p].begin(), byp[p].end());
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
  };
  std::vector<std::vector<int>> closure(N);
  for (int v = 0; v < nn; ++v)
    for (int J : R[v]) closure[J].push_back(v);
  // a coarse node of one part is that part's pressure column (P1-disc): a local set keeps it
  // only when the part is its own (the pressure of neighbouring parts is dropped with the rim)
  std::vector<char> own(nn, 0);
  bool any_own = false;
  for (int v = 0; v < nn; ++v) {
    own[v] = P.cn_set[v].size() == 1;
    any_own = any_own || own[v];
  }
  SlabSet& S = L.loc;
  S = SlabSet();
  std::vector<int> nb;
  for (int J = 0; J < N; ++J) {
    std::vector<char> in(nn, 0);
    for (int v : closure[J]) {
      in[v] = 1;
      neighbors(v, nb);
      for (int w : nb)
        if (!own[w]) in[w] = 1;
    }
    std::vector<int32_t> d;
    for (int v = 0; v < nn; ++v)
      if (in[v])
        for (int dd : P.cn_dofs[v]) d.push_back(dd);
    dense_order(d, S);
  }
  S.layout();
  scatter_lists(L, ctx->opt.weighting);
  // entities of this level
  std::map<std::vector<int>, int> gid;
  std::vector<int> grp(nn, -1);
  for (int v = 0; v < nn; ++v) {
    if (R[v].size() < 2) continue;
    auto it = gid.find(R[v]);
    if (it == gid.end()) it = gid.emplace(R[v], int(gid.size())).first;
    grp[v] = it->second;
  }
  struct Ent { std::vector<int> set; std::vector<int> nodes; };
  std::vector<Ent> ents;
  std::vector<char> seen(nn, 0);
  for (int v = 0; v < nn; ++v) {
    if (grp[v] < 0 || seen[v]) continue;
    Ent E;
    E.set = R[v];
    std::vector<int> stack{v};
    seen[v] = 1;
    while (!stack.empty()) {
      int a = stack.back();
      stack.pop_back();
      E.nodes.push_back(a);
      neighbors(a, nb);
      for (int w : nb)
        if (!seen[w] && grp[w] == grp[a]) {
          seen[w] = 1;
          stack.push_back(w);
        }
    }
    std::sort(E.nodes.begin(), E.nodes.end());
    ents.push_back(std::move(E));
  }
  std::sort(ents.begin(), ents.end(), [](const Ent& a, const Ent& b) {
    if (a.set != b.set) return a.set < b.set;
    return a.nodes[0] < b.nodes[0];
  });
  CoarseSpace& C = L.cs;
  C = CoarseSpace();
  C.n = L.n;
  C.nparts = N;
  C.n_entities = int(ents.size());
  int n0 = 0;
  std::vector<std::vector<int>> ent_cols(ents.size()), eset(ents.size());
  std::vector<std::pair<int32_t, int32_t>> gl;
  for (size_t e = 0; e < ents.size(); ++e) {
    bool present[4] = {false, false, false, false};
    for (int v : ents[e].nodes)
      for (int md : P.cn_modes[v]) present[md] = true;
    int col[4];
    std::vector<int> dofs, modes;
    for (int md = 0; md < 4; ++md) {
      col[md] = present[md] ? n0 : -1;
      if (present[md]) {
        dofs.push_back(n0);
        modes.push_back(md);
        ent_cols[e].push_back(n0);
        n0++;
      }
    }
    for (int v : ents[e].nodes)
      for (size_t q = 0; q < P.cn_dofs[v].size(); ++q) gl.push_back({P.cn_dofs[v][q], col[P.cn_modes[v][q]]});
    C.cn_set.push_back(ents[e].set);
    C.cn_dofs.push_back(dofs);
    C.cn_modes.push_back(modes);
    eset[e] = ents[e].set;
  }
  // P1-disc: one pressure column per part of this level, the sum of its members' pressure
  // columns, prescribed through them (they join Gamma); they become the next level's one-part
  // coarse nodes
  const bool pcols = any_own && N >= 2;
  if (pcols) {
    const int n_ent_cols = n0;
    for (int v = 0; v < nn; ++v)
      if (own[v])
        for (int dd : P.cn_dofs[v]) gl.push_back({dd, int32_t(n_ent_cols + R[v][0])});
    for (int J = 0; J < N; ++J) {
      C.cn_set.push_back({J});
      C.cn_dofs.push_back({n0});
      C.cn_modes.push_back({3});
      eset.push_back({J});
      ent_cols.push_back({n0});
      ++n0;
    }
  }
  C.n0 = n0;
  std::sort(gl.begin(), gl.end());
  for (auto& q : gl) {
    C.gdofs.push_back(q.first);
    C.gcol.push_back(q.second);
  }
  // interiors: nodes whose part set is {J} (not the part pressure nodes, which are in Gamma)
  SlabSet& I = L.inter;
  I = SlabSet();
  std::vector<std::vector<int32_t>> idof(N);
  for (int v = 0; v < nn; ++v)
    if (R[v].size() == 1 && !(pcols && own[v]))
      for (int dd : P.cn_dofs[v]) idof[R[v][0]].push_back(dd);
  for (int J = 0; J < N; ++J) dense_order(idof[J], I);
  I.layout();
  C.idofs = I.gdof;
  C.ioff = I.voff;
  coarse_lists(C, eset, ent_cols);
}

}  // namespace gdsw
