// Geometric multigrid with the multilevel GDSW method as its coarse-grid solver (arXiv
// 2606.01433, Section 3: besides preconditioning FGMRES, the Schwarz method solves the
// coarsest problem of a geometric multigrid method, by FGMRES to a relative residual of 1e-1).
//
// Grids are the contexts the caller set up, finest first, on one stream: every grid but the
// coarsest is an operator-only context (assembly, SpMV), the coarsest carries the multilevel
// GDSW preconditioner and its FGMRES tolerance (the coarse-solve tolerance).  The multigrid
// object adds, per fine grid:
//   * the element-Vanka patches: for every fluid element, the free dofs of its 27 Q2 and 8 Q1
//     nodes (at most 89, padded to 96) and the explicit inverse of the principal submatrix of
//     the assembled operator on them (extracted on the device, inverted in FP64, stored FP32
//     or FP64 column-major); elements coloured by the parity of their voxel indices, so the
//     patches of one colour are disjoint;
//   * the transfer to the next coarser grid: nodal interpolation P of the coarse Q2 velocity
//     and Q1 pressure at the fine nodes (zero correction at coarse Dirichlet nodes) and
//     R = P^T, both as CSR matrices built on the host;
// and attaches its V-cycle as the preconditioner of the finest context, so gdsw_solve on
// that context runs FP64 FGMRES preconditioned by the V-cycle:
//   V(l, b): z = 0; nu1 smoothing steps; b_{l+1} = R (b - A z); z += P V(l+1, b_{l+1});
//            nu2 smoothing steps; on the coarsest grid FGMRES + GDSW from zero.
// A smoothing step sweeps the eight colours: r = b - A z, then one warp per patch of the colour
// computes A_e^{-1} r_e and adds omega times it to z (no two patches of a colour share a dof, so
// the additions need no ordering).  FP64 smoothing forms r with the full FP64 SpMV; FP32
// smoothing forms it only on the rows the colour's patches touch (about (3/4)^3 of them), with
// an FP32 copy of the operator taken when the multigrid is created.
#include <algorithm>
#include <cmath>

#include "common.h"
#include "kernels.h"
#include "setup.h"

namespace gdsw {

void apply_precond(gdsw_ctx* c, const double* r, double* z, cudaStream_t s);
static thread_local std::string g_mg_create_error;  // why the last gdsw_mg_create of this thread failed

constexpr int PMAX = 96;  // padded patch size (27 x 3 velocity + 8 pressure dofs at most)

struct MgGrid {
  gdsw_ctx* ctx = nullptr;
  int64_t n = 0;
  // Vanka patches, sorted by colour
  int64_t npatch = 0;
  int64_t colour_off[9] = {0};
  int32_t* d_pdof = nullptr;   // npatch x PMAX dofs, -1 padding
  void* d_pinv = nullptr;      // npatch x PMAX x PMAX, column-major inverse (FP32 or FP64)
  double minpiv = 0;
  // FP32 smoothing: an FP32 copy of the operator's values (taken at creation) and, per colour,
  // the velocity-node and pressure rows its patches touch (the residual is formed there only)
  float *d_a32 = nullptr, *d_bt32 = nullptr, *d_b32 = nullptr;
  int32_t* d_rows = nullptr;   // per colour: velocity nodes, then pressure indices
  int64_t vrow_off[9] = {0}, prow_off[9] = {0};
  // transfer to the next coarser grid
  int64_t nc = 0;
  int32_t *d_p_ptr = nullptr, *d_p_col = nullptr, *d_r_ptr = nullptr, *d_r_col = nullptr;
  double *d_p_val = nullptr, *d_r_val = nullptr;
  // work vectors
  double *d_b = nullptr, *d_z = nullptr, *d_r = nullptr;
};

}  // namespace gdsw

struct gdsw_mg {
  std::string err;
  gdsw_mg_options opt{};
  std::vector<gdsw::MgGrid> g;
  gdsw::DevArena arena;
  cudaStream_t s = nullptr;
  int64_t coarse_solves = 0, coarse_iterations = 0;
  int64_t cycles = 0;
};

namespace gdsw {

// ------------------------------------------------------------------ host symbolic work
struct PatchHost {
  std::vector<int32_t> dof;  // npatch x PMAX
  int64_t off[9] = {0};
};

// patches of every fluid element (see the header), grouped by colour
static PatchHost build_patches(const MeshHost& M) {
  std::vector<int64_t> order[8];
  for (int64_t f = 0; f < int64_t(M.fluid.size()); ++f) {
    const int64_t e = M.fluid[f];
    const int ex = int(e % M.nx), ey = int((e / M.nx) % M.ny), ez = int(e / (int64_t(M.nx) * M.ny));
    order[(ex & 1) + 2 * (ey & 1) + 4 * (ez & 1)].push_back(e);
  }
  PatchHost P;
  int64_t np = 0;
  for (int c = 0; c < 8; ++c) {
    P.off[c] = np;
    np += int64_t(order[c].size());
  }
  P.off[8] = np;
  P.dof.assign(size_t(np) * PMAX, -1);
  int64_t q = 0;
  for (int c = 0; c < 8; ++c)
    for (int64_t e : order[c]) {
      const int ex = int(e % M.nx), ey = int((e / M.nx) % M.ny), ez = int(e / (int64_t(M.nx) * M.ny));
      std::vector<int32_t> d;
      for (int a2 = 0; a2 < 3; ++a2)
        for (int a1 = 0; a1 < 3; ++a1)
          for (int a0 = 0; a0 < 3; ++a0) {
            const int64_t node = (2 * ex + a0) + int64_t(M.NX) * ((2 * ey + a1) + int64_t(M.NY) * (2 * ez + a2));
            const int32_t v = M.vidx[node];
            if (v >= 0)
              for (int cc = 0; cc < 3; ++cc) d.push_back(3 * v + cc);
            if ((a0 | a1 | a2) % 2 == 0 && M.pidx[node] >= 0) d.push_back(int32_t(M.nu + M.pidx[node]));
          }
      std::sort(d.begin(), d.end());
      GDSW_CHECK(int(d.size()) <= PMAX, GDSW_ERR_INVALID_ARG, "Vanka patch larger than its padding");
      std::copy(d.begin(), d.end(), P.dof.begin() + size_t(q) * PMAX);
      ++q;
    }
  return P;
}

// per colour, the velocity nodes and pressure indices that its patches touch (sorted)
static void colour_rows(const MeshHost& M, const PatchHost& P, std::vector<int32_t>& rows, int64_t voff[9],
                        int64_t poff[9]) {
  rows.clear();
  std::vector<int32_t> vmark(size_t(M.nv), -1), pmark(size_t(M.np), -1);
  for (int c = 0; c < 8; ++c) {
    std::vector<int32_t> vr, pr;
    for (int64_t q = P.off[c]; q < P.off[c + 1]; ++q)
      for (int k = 0; k < PMAX; ++k) {
        const int32_t d = P.dof[size_t(q) * PMAX + k];
        if (d < 0) break;
        if (d < M.nu) {
          if (vmark[d / 3] != c) {
            vmark[d / 3] = c;
            vr.push_back(d / 3);
          }
        } else if (pmark[d - M.nu] != c) {
          pmark[d - M.nu] = c;
          pr.push_back(int32_t(d - M.nu));
        }
      }
    std::sort(vr.begin(), vr.end());
    std::sort(pr.begin(), pr.end());
    voff[c] = int64_t(rows.size());
    rows.insert(rows.end(), vr.begin(), vr.end());
    poff[c] = int64_t(rows.size());
    rows.insert(rows.end(), pr.begin(), pr.end());
  }
  voff[8] = poff[8] = int64_t(rows.size());
}

// quadratic Lagrange weights of the nodes 0, 1, 2 at t in [0, 2]
static void lagrange2(double t, double w[3]) {
  w[0] = (t - 1.0) * (t - 2.0) * 0.5;
  w[1] = t * (2.0 - t);
  w[2] = t * (t - 1.0) * 0.5;
}

// coarse Q2 node indices / weights along one axis for fine Q2 node index i (coarse mc elements)
static int axis_q2(int i, int mc, int idx[3], double w[3]) {
  const int E = std::min(i / 4, mc - 1);     // fine node i sits at coarse node coordinate i / 2
  double lw[3];
  lagrange2(0.5 * i - 2.0 * E, lw);
  int k = 0;
  for (int a = 0; a < 3; ++a)
    if (lw[a] != 0.0) {
      idx[k] = 2 * E + a;
      w[k++] = lw[a];
    }
  return k;
}

// coarse Q1 vertex indices / weights for fine Q1 index p (fine vertex p at coarse coordinate p/2)
static int axis_q1(int p, int mc, int idx[2], double w[2]) {
  const int P0 = std::min(p / 2, mc - 1);
  const double f = 0.5 * p - P0;
  int k = 0;
  if (1.0 - f != 0.0) {
    idx[k] = P0;
    w[k++] = 1.0 - f;
  }
  if (f != 0.0) {
    idx[k] = P0 + 1;
    w[k++] = f;
  }
  return k;
}

struct CsrHost {
  std::vector<int32_t> ptr, col;
  std::vector<double> val;
};

// P: coarse free dofs -> fine free dofs, rows in fine dof order
static CsrHost build_prolongation(const MeshHost& F, const MeshHost& C) {
  GDSW_CHECK(F.nx == 2 * C.nx && F.ny == 2 * C.ny && F.nz == 2 * C.nz, GDSW_ERR_INVALID_ARG,
             "multigrid grids must be nested (each twice as fine as the next)");
  for (int64_t e = 0; e < int64_t(F.nx) * F.ny * F.nz; ++e) {
    const int ex = int(e % F.nx), ey = int((e / F.nx) % F.ny), ez = int(e / (int64_t(F.nx) * F.ny));
    const int64_t ce = (ex / 2) + int64_t(C.nx) * ((ey / 2) + int64_t(C.ny) * (ez / 2));
    GDSW_CHECK(F.mask[e] == C.mask[ce], GDSW_ERR_INVALID_ARG, "fine grid is not the refinement of the coarse grid");
  }
  CsrHost P;
  P.ptr.assign(size_t(F.n) + 1, 0);
  std::vector<int32_t> cols;
  std::vector<double> vals;
  auto emit_velocity = [&](int64_t vf) {
    const int64_t node = F.vnode[vf];
    int i, j, k;
    F.coords(node, i, j, k);
    int I[3], J[3], K[3];
    double wi[3], wj[3], wk[3];
    const int ni = axis_q2(i, C.nx, I, wi), nj = axis_q2(j, C.ny, J, wj), nk = axis_q2(k, C.nz, K, wk);
    std::vector<std::pair<int32_t, double>> row;
    for (int a = 0; a < ni; ++a)
      for (int b = 0; b < nj; ++b)
        for (int d = 0; d < nk; ++d) {
          const int64_t cn = I[a] + int64_t(C.NX) * (J[b] + int64_t(C.NY) * K[d]);
          const int32_t vc = C.vidx[cn];
          if (vc >= 0) row.push_back({vc, wi[a] * wj[b] * wk[d]});
        }
    std::sort(row.begin(), row.end());
    return row;
  };
  for (int64_t vf = 0; vf < F.nv; ++vf) {
    auto row = emit_velocity(vf);
    for (int cc = 0; cc < 3; ++cc) {
      for (auto& kv : row) {
        cols.push_back(3 * kv.first + cc);
        vals.push_back(kv.second);
      }
      P.ptr[3 * vf + cc + 1] = int32_t(cols.size());
    }
  }
  for (int64_t pf = 0; pf < F.np; ++pf) {
    int i, j, k;
    F.coords(F.pnode[pf], i, j, k);
    int I[2], J[2], K[2];
    double wi[2], wj[2], wk[2];
    const int ni = axis_q1(i / 2, C.nx, I, wi), nj = axis_q1(j / 2, C.ny, J, wj), nk = axis_q1(k / 2, C.nz, K, wk);
    std::vector<std::pair<int32_t, double>> row;
    for (int a = 0; a < ni; ++a)
      for (int b = 0; b < nj; ++b)
        for (int d = 0; d < nk; ++d) {
          const int64_t cn = 2 * I[a] + int64_t(C.NX) * (2 * J[b] + int64_t(C.NY) * 2 * K[d]);
          const int32_t pc = C.pidx[cn];
          GDSW_CHECK(pc >= 0, GDSW_ERR_INVALID_ARG, "coarse pressure vertex outside the fluid");
          row.push_back({int32_t(C.nu + pc), wi[a] * wj[b] * wk[d]});
        }
    std::sort(row.begin(), row.end());
    for (auto& kv : row) {
      cols.push_back(kv.first);
      vals.push_back(kv.second);
    }
    P.ptr[F.nu + pf + 1] = int32_t(cols.size());
  }
  P.col = std::move(cols);
  P.val = std::move(vals);
  return P;
}

// R = P^T as CSR (rows = coarse dofs), entries of a row in increasing fine dof
static CsrHost transpose(const CsrHost& P, int64_t nc) {
  CsrHost R;
  R.ptr.assign(size_t(nc) + 1, 0);
  for (int32_t c : P.col) ++R.ptr[c + 1];
  for (int64_t r = 0; r < nc; ++r) R.ptr[r + 1] += R.ptr[r];
  R.col.resize(P.col.size());
  R.val.resize(P.val.size());
  std::vector<int32_t> fill(R.ptr.begin(), R.ptr.end() - 1);
  const int64_t nf = int64_t(P.ptr.size()) - 1;
  for (int64_t r = 0; r < nf; ++r)
    for (int32_t q = P.ptr[r]; q < P.ptr[r + 1]; ++q) {
      const int32_t c = P.col[q];
      R.col[fill[c]] = int32_t(r);
      R.val[fill[c]++] = P.val[q];
    }
  return R;
}

// ------------------------------------------------------------------ kernels
// dense copy of every patch's principal submatrix: A[row][col] for the patch dofs, read from
// the block operator (3 x 3 velocity blocks, B^T and B as 3-vectors); one CTA per patch
__global__ void k_patch_extract(const int32_t* __restrict__ pdof, int64_t npatch, MatView v, int64_t nu,
                                double* __restrict__ out) {
  const int64_t q = blockIdx.x;
  if (q >= npatch) return;
  const int32_t* d = pdof + q * PMAX;
  double* o = out + q * PMAX * PMAX;
  for (int t = threadIdx.x; t < PMAX * PMAX; t += blockDim.x) {
    const int i = t / PMAX, j = t % PMAX;  // row-major
    const int32_t di = d[i], dj = d[j];
    double val = 0.0;
    if (di >= 0 && dj >= 0) {
      if (di < nu && dj < nu) {
        const int32_t I = di / 3, J = dj / 3;
        int32_t lo = v.a_ptr[I], hi = v.a_ptr[I + 1] - 1;
        while (lo <= hi) {  // columns of a block row are sorted
          const int32_t mid = (lo + hi) >> 1, cm = v.a_col[mid];
          if (cm == J) {
            val = v.aval[int64_t(mid) * 9 + (di % 3) * 3 + (dj % 3)];
            break;
          }
          if (cm < J) lo = mid + 1; else hi = mid - 1;
        }
      } else if (di < nu) {  // velocity row, pressure column: B^T
        const int32_t I = di / 3, P = int32_t(dj - nu);
        for (int32_t e = v.bt_ptr[I]; e < v.bt_ptr[I + 1]; ++e)
          if (v.bt_col[e] == P) {
            val = v.btval[int64_t(e) * 3 + di % 3];
            break;
          }
      } else if (dj < nu) {  // pressure row, velocity column: B
        const int32_t P = int32_t(di - nu), J = dj / 3;
        for (int32_t e = v.b_ptr[P]; e < v.b_ptr[P + 1]; ++e)
          if (v.b_col[e] == J) {
            val = v.bval[int64_t(e) * 3 + dj % 3];
            break;
          }
      }
    }
    o[t] = val;
  }
}

// row-major FP64 inverse (n x n inside a PMAX x PMAX block) -> column-major, zero padded
template <typename TM>
__global__ void k_patch_store(const double* __restrict__ inv, const int32_t* __restrict__ pdof, int64_t npatch,
                              TM* __restrict__ out) {
  const int64_t q = blockIdx.x;
  if (q >= npatch) return;
  const int32_t* d = pdof + q * PMAX;
  for (int t = threadIdx.x; t < PMAX * PMAX; t += blockDim.x) {
    const int col = t / PMAX, row = t % PMAX;  // column-major position t
    const bool in = d[row] >= 0 && d[col] >= 0;
    out[q * PMAX * PMAX + t] = in ? TM(inv[q * PMAX * PMAX + int64_t(row) * PMAX + col]) : TM(0);
  }
}

// one warp per patch of a colour: z[d] += omega A_e^{-1} r[d]; lane owns rows lane + 32 k
template <typename TM>
__global__ void __launch_bounds__(256) k_vanka(const int32_t* __restrict__ pdof, const TM* __restrict__ pinv,
                                               int64_t p0, int64_t p1, const double* __restrict__ r,
                                               double* __restrict__ z, double omega) {
  const int64_t q = p0 + (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  dep_release();
  if (q < p1)  // the patch inverse is set-up data: its first 4 KB go to L2 before the wait
    prefetch_l2(reinterpret_cast<const char*>(pinv + q * PMAX * PMAX) + 128 * lane);
  dep_wait();
  if (q >= p1) return;
  const int32_t* d = pdof + q * PMAX;
  const TM* M = pinv + q * PMAX * PMAX;
  int32_t dof[3];
  TM rv[3], y[3] = {TM(0), TM(0), TM(0)};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dof[k] = d[lane + 32 * k];
    rv[k] = dof[k] >= 0 ? TM(r[dof[k]]) : TM(0);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll 8
    for (int jj = 0; jj < 32; ++jj) {
      const TM rj = __shfl_sync(0xffffffffu, rv[k], jj);
      const TM* col = M + int64_t(32 * k + jj) * PMAX;
#pragma unroll
      for (int u = 0; u < 3; ++u) y[u] = fma(__ldcs(col + lane + 32 * u), rj, y[u]);
    }
#pragma unroll
  for (int u = 0; u < 3; ++u)
    if (dof[u] >= 0) z[dof[u]] += omega * double(y[u]);
}

// r = b - A z on the velocity-node rows of a list, FP32 operator values and products, FP64
// b and result: one warp per node, lanes over its 3x3 blocks and B^T entries, fixed butterfly
__global__ void __launch_bounds__(256) k_resid_vrows(const int32_t* __restrict__ rows, int64_t nrows,
                                                     const int32_t* __restrict__ a_ptr,
                                                     const int32_t* __restrict__ a_col, const float* __restrict__ a32,
                                                     const int32_t* __restrict__ bt_ptr,
                                                     const int32_t* __restrict__ bt_col,
                                                     const float* __restrict__ bt32, int64_t nu,
                                                     const double* __restrict__ z, const double* __restrict__ b,
                                                     double* __restrict__ r) {
  const int64_t q = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  dep_release();
  dep_wait();
  if (q >= nrows) return;
  const int32_t I = rows[q];
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int32_t e = a_ptr[I] + lane; e < a_ptr[I + 1]; e += 32) {
    const int64_t J = a_col[e];
    const float x0 = float(z[3 * J]), x1 = float(z[3 * J + 1]), x2 = float(z[3 * J + 2]);
    const float* v = a32 + int64_t(e) * 9;
    s0 = fmaf(v[0], x0, fmaf(v[1], x1, fmaf(v[2], x2, s0)));
    s1 = fmaf(v[3], x0, fmaf(v[4], x1, fmaf(v[5], x2, s1)));
    s2 = fmaf(v[6], x0, fmaf(v[7], x1, fmaf(v[8], x2, s2)));
  }
  for (int32_t e = bt_ptr[I] + lane; e < bt_ptr[I + 1]; e += 32) {
    const float xp = float(z[nu + bt_col[e]]);
    const float* v = bt32 + int64_t(e) * 3;
    s0 = fmaf(v[0], xp, s0);
    s1 = fmaf(v[1], xp, s1);
    s2 = fmaf(v[2], xp, s2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane < 3) {
    const int64_t d = 3 * int64_t(I) + lane;
    r[d] = b[d] - double(lane == 0 ? s0 : (lane == 1 ? s1 : s2));
  }
}

// r = b - A z on the pressure rows of a list (FP32 values and products): one warp per row
__global__ void __launch_bounds__(256) k_resid_prows(const int32_t* __restrict__ rows, int64_t nrows,
                                                     const int32_t* __restrict__ b_ptr,
                                                     const int32_t* __restrict__ b_col, const float* __restrict__ b32,
                                                     int64_t nu, const double* __restrict__ z,
                                                     const double* __restrict__ b, double* __restrict__ r) {
  const int64_t q = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  dep_release();
  dep_wait();
  if (q >= nrows) return;
  const int32_t P = rows[q];
  float s = 0.f;
  for (int32_t e = b_ptr[P] + lane; e < b_ptr[P + 1]; e += 32) {
    const int64_t J = b_col[e];
    const float* v = b32 + int64_t(e) * 3;
    s = fmaf(v[0], float(z[3 * J]), fmaf(v[1], float(z[3 * J + 1]), fmaf(v[2], float(z[3 * J + 2]), s)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) r[nu + P] = b[nu + P] - double(s);
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) b[i] = float(a[i]);
}

// y = M x (+ y when accumulate), CSR FP64, one thread per row
__global__ void k_csr_mv(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                         const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                         int64_t n, int accumulate) {
  const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  dep_release();
  dep_wait();
  if (r >= n) return;
  double acc = accumulate ? y[r] : 0.0;
  for (int32_t q = ptr[r]; q < ptr[r + 1]; ++q) acc = fma(val[q], x[col[q]], acc);
  y[r] = acc;
}

static void csr_mv(const int32_t* ptr, const int32_t* col, const double* val, const double* x, double* y, int64_t n,
                   bool acc, cudaStream_t s) {
  if (n == 0) return;
  launch_chained(k_csr_mv, dim3(unsigned((n + 255) / 256)), dim3(256), 0, s, ptr, col, val, x, y, n, acc ? 1 : 0);
  check_launch("k_csr_mv");
}

// ------------------------------------------------------------------ the cycle
// r = b - A z where colour c's patches need it: the full FP64 SpMV for FP64 smoothing, the
// colour's rows in FP32 products otherwise
static void colour_residual(gdsw_mg* mg, MgGrid& G, int c, const double* b, const double* z, cudaStream_t s) {
  if (mg->opt.smoother_precision == GDSW_FP64) {
    launch_spmv(G.ctx, z, G.d_r, b, s);
    return;
  }
  const gdsw_ctx* x = G.ctx;
  const int64_t nv = G.prow_off[c] - G.vrow_off[c], np = G.vrow_off[c + 1] - G.prow_off[c];
  if (nv > 0) {
    launch_chained(k_resid_vrows, dim3(unsigned((nv + 7) / 8)), dim3(256), 0, s, G.d_rows + G.vrow_off[c], nv,
                   x->d_a_ptr, x->d_a_col, G.d_a32, x->d_bt_ptr, x->d_bt_col, G.d_bt32, x->mesh.nu, z, b, G.d_r);
    check_launch("k_resid_vrows");
  }
  if (np > 0) {
    launch_chained(k_resid_prows, dim3(unsigned((np + 7) / 8)), dim3(256), 0, s, G.d_rows + G.prow_off[c], np,
                   x->d_b_ptr, x->d_b_col, G.d_b32, x->mesh.nu, z, b, G.d_r);
    check_launch("k_resid_prows");
  }
}

// reverse: sweep the colours 7..0 (the post-smoothing of a symmetric cycle)
static void smooth(gdsw_mg* mg, int l, const double* b, double* z, int steps, bool reverse = false) {
  MgGrid& G = mg->g[l];
  cudaStream_t s = mg->s;
  for (int it = 0; it < steps; ++it)
    for (int cc = 0; cc < 8; ++cc) {
      const int c = reverse ? 7 - cc : cc;
      const int64_t p0 = G.colour_off[c], p1 = G.colour_off[c + 1];
      if (p1 == p0) continue;
      colour_residual(mg, G, c, b, z, s);
      const int blocks = int((p1 - p0 + 7) / 8);
      if (mg->opt.smoother_precision == GDSW_FP64)
        launch_chained(k_vanka<double>, dim3(unsigned(blocks)), dim3(256), 0, s, G.d_pdof,
                       static_cast<const double*>(G.d_pinv), p0, p1, G.d_r, z, mg->opt.omega);
      else
        launch_chained(k_vanka<float>, dim3(unsigned(blocks)), dim3(256), 0, s, G.d_pdof,
                       static_cast<const float*>(G.d_pinv), p0, p1, G.d_r, z, mg->opt.omega);
      check_launch("k_vanka");
    }
}

static void vcycle(gdsw_mg* mg, int l, const double* b, double* z) {
  cudaStream_t s = mg->s;
  MgGrid& G = mg->g[l];
  GDSW_CUDA(cudaMemsetAsync(z, 0, 8 * G.n, s));
  if (l + 1 == int(mg->g.size())) {  // coarsest grid: FGMRES + multilevel GDSW from zero
    gdsw_solve_info info{};
    fgmres_solve(G.ctx, b, z, &info);
    GDSW_CHECK(info.status == GDSW_OK || info.status == GDSW_ERR_NOT_CONVERGED, info.status,
               "coarse-grid solve failed: " + G.ctx->err);
    ++mg->coarse_solves;
    mg->coarse_iterations += info.iterations;
    return;
  }
  MgGrid& C = mg->g[l + 1];
  smooth(mg, l, b, z, mg->opt.pre);
  launch_spmv(G.ctx, z, G.d_r, b, s);                                      // r = b - A z
  csr_mv(G.d_r_ptr, G.d_r_col, G.d_r_val, G.d_r, C.d_b, G.nc, false, s);   // b_c = R r
  vcycle(mg, l + 1, C.d_b, C.d_z);
  csr_mv(G.d_p_ptr, G.d_p_col, G.d_p_val, C.d_z, z, G.n, true, s);         // z += P z_c
  smooth(mg, l, b, z, mg->opt.post, mg->opt.symmetric != 0);
}

static void mg_precond(void* data, const double* r, double* z, cudaStream_t s) {
  gdsw_mg* mg = static_cast<gdsw_mg*>(data);
  (void)s;
  ++mg->cycles;
  vcycle(mg, 0, r, z);
}

static void mg_create(gdsw_mg* mg, gdsw_ctx* const* grids, int ngrids, const gdsw_mg_options* opt) {
  GDSW_CHECK(grids && opt && ngrids >= 2 && ngrids <= 8, GDSW_ERR_INVALID_ARG, "need 2 to 8 grids");
  GDSW_CHECK(opt->pre >= 0 && opt->post >= 0 && opt->pre + opt->post > 0 && opt->omega > 0, GDSW_ERR_INVALID_ARG,
             "bad smoothing parameters");
  GDSW_CHECK(opt->smoother_precision == GDSW_FP64 || opt->smoother_precision == GDSW_FP32, GDSW_ERR_INVALID_ARG,
             "smoother precision must be FP64 or FP32");
  mg->opt = *opt;
  mg->s = grids[0] ? grids[0]->stream : nullptr;
  for (int l = 0; l < ngrids; ++l) {
    gdsw_ctx* c = grids[l];
    GDSW_CHECK(c && !c->host_only, GDSW_ERR_INVALID_ARG, "null or analysis-only grid context");
    GDSW_CHECK(c->stream == mg->s, GDSW_ERR_INVALID_ARG, "all grid contexts must use one stream");
    GDSW_CHECK((l + 1 == ngrids) == (c->L >= 2), GDSW_ERR_INVALID_ARG,
               "fine grids must be operator-only contexts (levels = 1), the coarsest a GDSW context");
    GDSW_CHECK(!c->ext_precond, GDSW_ERR_INVALID_ARG, "grid context already has a multigrid attached");
    GDSW_CHECK(!c->mesh.pdisc, GDSW_ERR_INVALID_ARG, "the multigrid transfers are defined for Q1 pressure");
  }
  cudaStream_t s = mg->s;
  mg->arena.stream = s;
  mg->arena.ordered = true;
  mg->g.resize(ngrids);
  for (int l = 0; l < ngrids; ++l) {
    MgGrid& G = mg->g[l];
    G.ctx = grids[l];
    G.n = G.ctx->mesh.n;
    G.d_b = mg->arena.alloc<double>(G.n);
    G.d_z = mg->arena.alloc<double>(G.n);
    G.d_r = mg->arena.alloc<double>(G.n);
  }
  for (int l = 0; l + 1 < ngrids; ++l) {
    MgGrid& G = mg->g[l];
    const MeshHost& M = G.ctx->mesh;
    // patches and their inverses
    PatchHost P = build_patches(M);
    G.npatch = P.off[8];
    std::copy(P.off, P.off + 9, G.colour_off);
    G.d_pdof = mg->arena.upload(P.dof, s);
    DevArena tmp(s);
    try {
      double* dense = tmp.alloc<double>(size_t(G.npatch) * PMAX * PMAX);
      MatView v;
      v.n = M.n;
      v.nu = M.nu;
      v.a_ptr = G.ctx->d_a_ptr;
      v.a_col = G.ctx->d_a_col;
      v.bt_ptr = G.ctx->d_bt_ptr;
      v.bt_col = G.ctx->d_bt_col;
      v.b_ptr = G.ctx->d_b_ptr;
      v.b_col = G.ctx->d_b_col;
      v.aval = G.ctx->d_val;
      v.btval = G.ctx->d_val + 9 * G.ctx->nnzb;
      v.bval = v.btval + 3 * G.ctx->nbt;
      if (G.npatch > 0) {
        k_patch_extract<<<unsigned(G.npatch), 256, 0, s>>>(G.d_pdof, G.npatch, v, M.nu, dense);
        check_launch("k_patch_extract");
      }
      std::vector<InvTaskP> inv;
      inv.reserve(size_t(G.npatch));
      for (int64_t q = 0; q < G.npatch; ++q) {
        int n = 0;
        while (n < PMAX && P.dof[size_t(q) * PMAX + n] >= 0) ++n;
        inv.push_back({dense + q * PMAX * PMAX, n, PMAX, 0});
      }
      G.minpiv = 1e300;
      constexpr size_t kChunk = 32768;  // the batched inverse puts tasks on a grid axis of <= 65535
      for (size_t i0 = 0; i0 < inv.size(); i0 += kChunk) {
        std::vector<InvTaskP> part(inv.begin() + i0, inv.begin() + std::min(inv.size(), i0 + kChunk));
        std::vector<double> mp;
        run_inverse<double>(tmp, part, mp, s);
        for (double x : mp) G.minpiv = std::min(G.minpiv, x);
      }
      GDSW_CHECK(G.minpiv > 0 && std::isfinite(G.minpiv), GDSW_ERR_SINGULAR, "Vanka patch matrix is singular");
      if (opt->smoother_precision == GDSW_FP64) {
        double* st = mg->arena.alloc<double>(size_t(G.npatch) * PMAX * PMAX);
        if (G.npatch) k_patch_store<double><<<unsigned(G.npatch), 256, 0, s>>>(dense, G.d_pdof, G.npatch, st);
        G.d_pinv = st;
      } else {
        float* st = mg->arena.alloc<float>(size_t(G.npatch) * PMAX * PMAX);
        if (G.npatch) k_patch_store<float><<<unsigned(G.npatch), 256, 0, s>>>(dense, G.d_pdof, G.npatch, st);
        G.d_pinv = st;
      }
      if (G.npatch) check_launch("k_patch_store");
      GDSW_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      tmp.free_all();
      throw;
    }
    tmp.free_all();
    if (opt->smoother_precision == GDSW_FP32) {
      std::vector<int32_t> rows;
      colour_rows(M, P, rows, G.vrow_off, G.prow_off);
      G.d_rows = mg->arena.upload(rows, s);
      const gdsw_ctx* x = G.ctx;
      const int64_t na = 9 * x->nnzb, nbt = 3 * x->nbt, nb = 3 * x->nb;
      G.d_a32 = mg->arena.alloc<float>(na);
      G.d_bt32 = mg->arena.alloc<float>(nbt);
      G.d_b32 = mg->arena.alloc<float>(nb);
      k_to_f32<<<int((na + 255) / 256), 256, 0, s>>>(x->d_val, G.d_a32, na);
      k_to_f32<<<int((nbt + 255) / 256), 256, 0, s>>>(x->d_val + na, G.d_bt32, nbt);
      k_to_f32<<<int((nb + 255) / 256), 256, 0, s>>>(x->d_val + na + nbt, G.d_b32, nb);
      check_launch("k_to_f32");
    }
    // transfers
    const MeshHost& Cm = mg->g[l + 1].ctx->mesh;
    CsrHost Ph = build_prolongation(M, Cm);
    CsrHost Rh = transpose(Ph, Cm.n);
    G.nc = Cm.n;
    G.d_p_ptr = mg->arena.upload(Ph.ptr, s);
    G.d_p_col = mg->arena.upload(Ph.col, s);
    G.d_p_val = mg->arena.upload(Ph.val, s);
    G.d_r_ptr = mg->arena.upload(Rh.ptr, s);
    G.d_r_col = mg->arena.upload(Rh.col, s);
    G.d_r_val = mg->arena.upload(Rh.val, s);
  }
  GDSW_CUDA(cudaStreamSynchronize(s));
  grids[0]->ext_precond = mg_precond;
  grids[0]->ext_data = mg;
}

}  // namespace gdsw

using namespace gdsw;

#define MG_TRY(mg, body)                  \
  try {                                   \
    body;                                 \
    return GDSW_OK;                       \
  } catch (const gdsw::Error& e) {        \
    (mg)->err = e.msg;                    \
    return e.code;                        \
  } catch (const std::bad_alloc&) {       \
    (mg)->err = "host allocation failed"; \
    return GDSW_ERR_OOM;                  \
  } catch (...) {                         \
    (mg)->err = "unknown error";          \
    return GDSW_ERR_CUDA;                 \
  }

extern "C" {

int gdsw_mg_create(gdsw_ctx* const* grids, int32_t ngrids, const gdsw_mg_options* opt, gdsw_mg** out) {
  if (!out) return GDSW_ERR_INVALID_ARG;
  *out = nullptr;
  gdsw_mg* mg = new (std::nothrow) gdsw_mg();
  if (!mg) return GDSW_ERR_OOM;
  int rc = GDSW_OK;
  try {
    mg_create(mg, grids, ngrids, opt);
  } catch (const gdsw::Error& e) {
    mg->err = e.msg;
    rc = e.code;
  } catch (const std::bad_alloc&) {
    mg->err = "host allocation failed";
    rc = GDSW_ERR_OOM;
  } catch (...) {
    mg->err = "unknown error";
    rc = GDSW_ERR_CUDA;
  }
  if (rc != GDSW_OK) {
    g_mg_create_error = mg->err;
    mg->arena.free_all();
    if (mg->s) cudaStreamSynchronize(mg->s);
    delete mg;
    return rc;
  }
  *out = mg;
  return GDSW_OK;
}

void gdsw_mg_destroy(gdsw_mg* mg) {
  if (!mg) return;
  if (!mg->g.empty() && mg->g[0].ctx && mg->g[0].ctx->ext_data == mg) {
    mg->g[0].ctx->ext_precond = nullptr;
    mg->g[0].ctx->ext_data = nullptr;
  }
  mg->arena.free_all();
  if (mg->s) cudaStreamSynchronize(mg->s);
  delete mg;
}

const char* gdsw_mg_last_error(const gdsw_mg* mg) { return mg ? mg->err.c_str() : g_mg_create_error.c_str(); }

int gdsw_mg_vcycle(gdsw_mg* mg, const double* r, double* z) {
  if (!mg || !r || !z) return GDSW_ERR_INVALID_ARG;
  MG_TRY(mg, vcycle(mg, 0, r, z));
}

int gdsw_mg_smooth(gdsw_mg* mg, int32_t grid, const double* b, double* x, int32_t steps) {
  if (!mg || !b || !x || grid < 0 || grid + 1 >= int(mg->g.size()) || steps < 0) return GDSW_ERR_INVALID_ARG;
  MG_TRY(mg, smooth(mg, grid, b, x, steps));
}

int gdsw_mg_prolong(gdsw_mg* mg, int32_t grid, const double* xc, double* zf) {
  if (!mg || !xc || !zf || grid < 0 || grid + 1 >= int(mg->g.size())) return GDSW_ERR_INVALID_ARG;
  const MgGrid& G = mg->g[grid];
  MG_TRY(mg, csr_mv(G.d_p_ptr, G.d_p_col, G.d_p_val, xc, zf, G.n, true, mg->s));
}

int gdsw_mg_restrict(gdsw_mg* mg, int32_t grid, const double* rf, double* rc) {
  if (!mg || !rf || !rc || grid < 0 || grid + 1 >= int(mg->g.size())) return GDSW_ERR_INVALID_ARG;
  const MgGrid& G = mg->g[grid];
  MG_TRY(mg, csr_mv(G.d_r_ptr, G.d_r_col, G.d_r_val, rf, rc, G.nc, false, mg->s));
}

int gdsw_mg_stats(const gdsw_mg* mg, int64_t* cycles, int64_t* coarse_solves, int64_t* coarse_iterations) {
  if (!mg) return GDSW_ERR_INVALID_ARG;
  if (cycles) *cycles = mg->cycles;
  if (coarse_solves) *coarse_solves = mg->coarse_solves;
  if (coarse_iterations) *coarse_iterations = mg->coarse_iterations;
  return GDSW_OK;
}

}  // extern "C"
