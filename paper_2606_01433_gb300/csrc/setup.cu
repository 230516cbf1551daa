// Device kernels of the numeric set-up (arXiv 2606.01433, Section 2.1 and 2.2):
//  - extraction of the local saddle-point matrices A_i = R_i A R_i^T into the blocks of a
//    block-tridiagonal (slab) ordering: diagonal blocks, and the sub/super-diagonal
//    couplings restricted to the back-coupled dofs;
//  - the right-hand sides -A_IGamma Phi_Gamma of the coarse-basis extension, and the
//    pieces of the Galerkin product A_0 = Phi^T A Phi;
//  - dense gathers and basis assembly on the coarse levels.
#include "common.h"
#include "kernels.h"
#include "setup.h"

namespace gdsw {

// visit the nonzeros of global row g: f(col, value)
template <typename F>
__device__ __forceinline__ void row_visit(const MatView& A, int64_t g, F f) {
  if (g < A.nu) {
    int64_t I = g / 3;
    int c = int(g - 3 * I);
    for (int blk = A.a_ptr[I]; blk < A.a_ptr[I + 1]; ++blk) {
      int64_t J = A.a_col[blk];
      const double* v = A.aval + int64_t(blk) * 9 + c * 3;
      f(3 * J + 0, v[0]);
      f(3 * J + 1, v[1]);
      f(3 * J + 2, v[2]);
    }
    for (int e = A.bt_ptr[I]; e < A.bt_ptr[I + 1]; ++e) f(A.nu + A.bt_col[e], A.btval[int64_t(e) * 3 + c]);
  } else {
    int64_t P = g - A.nu;
    for (int e = A.b_ptr[P]; e < A.b_ptr[P + 1]; ++e) {
      int64_t J = A.b_col[e];
      const double* v = A.bval + int64_t(e) * 3;
      f(3 * J + 0, v[0]);
      f(3 * J + 1, v[1]);
      f(3 * J + 2, v[2]);
    }
  }
}

__global__ void k_map_set(const int32_t* __restrict__ gdof, const int32_t* __restrict__ owner, int64_t p0, int64_t p1,
                          int i0, int separate, int64_t n, int32_t* __restrict__ map) {
  int64_t p = p0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p >= p1) return;
  int64_t slot = separate ? int64_t(owner[p] - i0) * n : 0;
  map[slot + gdof[p]] = int32_t(p);
}

__global__ void k_map_reset(const int32_t* __restrict__ gdof, const int32_t* __restrict__ owner, int64_t p0,
                            int64_t p1, int i0, int separate, int64_t n, int32_t* __restrict__ map) {
  int64_t p = p0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p >= p1) return;
  int64_t slot = separate ? int64_t(owner[p] - i0) * n : 0;
  map[slot + gdof[p]] = -1;
}

// Write A restricted to a slab set into its blocks: diagonal S_k, sub-diagonal B_k (rows
// = back-coupled dofs of slab k) and super-diagonal C_k (columns = back-coupled dofs of
// slab k+1).  Any other coupling means the ordering is wrong: flagged in *err.
template <typename T>
__global__ void k_extract(MatView A, SlabView S, int64_t p0, int64_t p1, int i0, int separate,
                          const int32_t* __restrict__ map, T* __restrict__ fac, int* __restrict__ err) {
  int64_t p = p0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p >= p1) return;
  const int i = S.owner[p];
  const int64_t slot = separate ? int64_t(i - i0) * A.n : 0;
  const int kr = S.pslab[p], r = S.pidx[p];
  const int sb = S.slab_base[i];
  row_visit(A, S.gdof[p], [&](int64_t col, double v) {
    int32_t q = map[slot + col];
    if (q < 0 || S.owner[q] != i) return;
    const int kc = S.pslab[q], c = S.pidx[q];
    if (kc == kr) {
      fac[S.fS[sb + kr] + int64_t(r) * S.ldS[sb + kr] + c] = T(v);
    } else if (kc == kr - 1 && r < S.m[sb + kr]) {
      fac[S.fG[sb + kr] + int64_t(r) * S.ldG[sb + kr] + c] = T(v);
    } else if (kc == kr + 1 && c < S.m[sb + kc]) {
      // super-diagonal coupling: the transpose of the next slab's sub-diagonal block
      if (S.fW[sb + kr] >= 0) fac[S.fW[sb + kr] + int64_t(r) * S.ldW[sb + kr] + c] = T(v);
    } else {
      atomicExch(err, 1);
    }
  });
}

template <typename T>
void extract_slabs(const MatView& A, const SlabView& S, int64_t p0, int64_t p1, int i0, int separate,
                   const int32_t* map, T* fac, int* err, cudaStream_t s) {
  if (p1 <= p0) return;
  int blocks = int((p1 - p0 + 127) / 128);
  k_map_set<<<blocks, 128, 0, s>>>(S.gdof, S.owner, p0, p1, i0, separate, A.n, const_cast<int32_t*>(map));
  k_extract<T><<<blocks, 128, 0, s>>>(A, S, p0, p1, i0, separate, map, fac, err);
  k_map_reset<<<blocks, 128, 0, s>>>(S.gdof, S.owner, p0, p1, i0, separate, A.n, const_cast<int32_t*>(map));
  check_launch("extract_slabs");
}
template void extract_slabs<double>(const MatView&, const SlabView&, int64_t, int64_t, int, int, const int32_t*,
                                    double*, int*, cudaStream_t);
template void extract_slabs<float>(const MatView&, const SlabView&, int64_t, int64_t, int, int, const int32_t*,
                                   float*, int*, cudaStream_t);

__device__ __forceinline__ int find_col(const int32_t* cols, int c, int key) {
  int lo = 0, hi = c;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cols[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return (lo < c && cols[lo] == key) ? lo : -1;
}

// Tneg = -A_IGamma Phi_Gamma for every interior row (one thread per row, nonzero order): each
// interface column adds its value times its Phi_Gamma entries (gamma_ptr: entry range of every
// dof, empty off the interface) to their coarse columns.
__global__ void k_tneg(MatView A, SlabView S, const int32_t* __restrict__ gamma_ptr, const int32_t* __restrict__ gcol,
                       const double* __restrict__ gval, const int32_t* __restrict__ cols,
                       const int64_t* __restrict__ coff, const int64_t* __restrict__ toff, const int32_t* __restrict__ ldt,
                       double* __restrict__ T, int* __restrict__ err) {
  int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p >= S.nvec) return;
  const int i = S.owner[p];
  const int64_t rowoff = toff[i] + (p - S.voff[i]) * ldt[i];
  const int32_t* ci = cols + coff[i];
  const int c = int(coff[i + 1] - coff[i]);
  row_visit(A, S.gdof[p], [&](int64_t col, double v) {
    for (int32_t e = gamma_ptr[col]; e < gamma_ptr[col + 1]; ++e) {
      int j = find_col(ci, c, gcol[e]);
      if (j < 0) {
        atomicExch(err, 2);
        return;
      }
      T[rowoff + j] -= v * gval[e];
    }
  });
}

// Y = A_II X - Tneg for interior rows (X = Phi_I, FP64): one warp per row, lanes over
// the coarse columns.  ilocal[g] = position of interior dof g in the concatenated
// interior vector (or -1).
__global__ void k_yint(MatView A, SlabView S, const int32_t* __restrict__ ilocal, const int64_t* __restrict__ coff,
                       const int64_t* __restrict__ toff, const int32_t* __restrict__ ldt, const double* __restrict__ X,
                       const double* __restrict__ Tn, double* __restrict__ Y) {
  int64_t p = blockIdx.x * int64_t(blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (p >= S.nvec) return;
  const int i = S.owner[p];
  const int c = int(coff[i + 1] - coff[i]);
  const int ld = ldt[i];
  const int64_t rowoff = toff[i] + (p - S.voff[i]) * ld;
  for (int j0 = 0; j0 < c; j0 += 32 * 4) {
    double acc[4] = {0, 0, 0, 0};
    row_visit(A, S.gdof[p], [&](int64_t col, double v) {
      int32_t q = ilocal[col];
      if (q < 0 || S.owner[q] != i) return;
      const double* xr = X + toff[i] + (q - S.voff[i]) * ld;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int j = j0 + lane + 32 * u;
        if (j < c) acc[u] = fma(v, xr[j], acc[u]);
      }
    });
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int j = j0 + lane + 32 * u;
      if (j < c) Y[rowoff + j] = acc[u] - Tn[rowoff + j];
    }
  }
}

// A0[key] += sum of (w *) src[pos] over a segment (deterministic list order; w null = 1)
__global__ void k_segsum(const int64_t* __restrict__ key, const int64_t* __restrict__ ptr,
                         const int64_t* __restrict__ pos, const double* __restrict__ w, int64_t nseg,
                         const double* __restrict__ src, double* __restrict__ dst) {
  int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (s >= nseg) return;
  double acc = 0.0;
  if (w)
    for (int64_t e = ptr[s]; e < ptr[s + 1]; ++e) acc = fma(w[e], src[pos[e]], acc);
  else
    for (int64_t e = ptr[s]; e < ptr[s + 1]; ++e) acc += src[pos[e]];
  dst[key[s]] += acc;
}

void segsum(const int64_t* key, const int64_t* ptr, const int64_t* pos, const double* w, int64_t nseg,
            const double* src, double* dst, cudaStream_t s) {
  if (nseg == 0) return;
  k_segsum<<<int((nseg + 255) / 256), 256, 0, s>>>(key, ptr, pos, w, nseg, src, dst);
  check_launch("k_segsum");
}

// ------------------------------------------------------------------ dense helpers (coarse levels)
// out_J[r][c] = A[d_J[r]][d_J[c]] (principal submatrix), written in precision T.
template <typename T>
__global__ void k_gather_dense(const double* __restrict__ A, int64_t n, const int32_t* __restrict__ dofs,
                               const int64_t* __restrict__ doff, const int32_t* __restrict__ part_of_row,
                               int64_t nrows, const int64_t* __restrict__ out_off, const int32_t* __restrict__ out_ld,
                               T* __restrict__ out) {
  int64_t row = blockIdx.x;
  if (row >= nrows) return;
  int J = part_of_row[row];
  int64_t r = row - doff[J];
  int sz = int(doff[J + 1] - doff[J]);
  const double* arow = A + int64_t(dofs[doff[J] + r]) * n;
  T* o = out + out_off[J] + r * out_ld[J];
  for (int c = threadIdx.x; c < sz; c += blockDim.x) o[c] = T(arow[dofs[doff[J] + c]]);
}

template <typename T>
void gather_dense(const double* A, int64_t n, const int32_t* dofs, const int64_t* doff, const int32_t* part_of_row,
                  int64_t nrows, const int64_t* out_off, const int32_t* out_ld, T* out, cudaStream_t s) {
  if (nrows == 0) return;
  k_gather_dense<T><<<int(nrows), 128, 0, s>>>(A, n, dofs, doff, part_of_row, nrows, out_off, out_ld, out);
  check_launch("k_gather_dense");
}
template void gather_dense<double>(const double*, int64_t, const int32_t*, const int64_t*, const int32_t*, int64_t,
                                   const int64_t*, const int32_t*, double*, cudaStream_t);
template void gather_dense<float>(const double*, int64_t, const int32_t*, const int64_t*, const int32_t*, int64_t,
                                  const int64_t*, const int32_t*, float*, cudaStream_t);

// Coarse-level Tneg_J[r][j] = -sum over interface dofs b of column cols_J[j] of A[I_J[r]][b]
__global__ void k_coarse_tneg(const double* __restrict__ A, int64_t n, const int32_t* __restrict__ idofs,
                              const int64_t* __restrict__ ioff, const int32_t* __restrict__ part_of_row, int64_t nrows,
                              const int32_t* __restrict__ gdofs, const int32_t* __restrict__ gcol, int64_t ng,
                              const int32_t* __restrict__ cols, const int64_t* __restrict__ coff,
                              const int64_t* __restrict__ toff, const int32_t* __restrict__ ldt, double* __restrict__ T) {
  int64_t row = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (row >= nrows) return;
  int J = part_of_row[row];
  int64_t r = row - ioff[J];
  const double* arow = A + int64_t(idofs[row]) * n;
  const int32_t* cj = cols + coff[J];
  int c = int(coff[J + 1] - coff[J]);
  double* t = T + toff[J] + r * ldt[J];
  for (int64_t q = 0; q < ng; ++q) {
    double v = arow[gdofs[q]];
    if (v == 0.0) continue;
    int j = find_col(cj, c, gcol[q]);
    if (j >= 0) t[j] -= v;
  }
}

void coarse_tneg(const double* A, int64_t n, const int32_t* idofs, const int64_t* ioff, const int32_t* part_of_row,
                 int64_t nrows, const int32_t* gdofs, const int32_t* gcol, int64_t ng, const int32_t* cols,
                 const int64_t* coff, const int64_t* toff, const int32_t* ldt, double* T, cudaStream_t s) {
  if (nrows == 0) return;
  k_coarse_tneg<<<int((nrows + 127) / 128), 128, 0, s>>>(A, n, idofs, ioff, part_of_row, nrows, gdofs, gcol, ng, cols,
                                                         coff, toff, ldt, T);
  check_launch("k_coarse_tneg");
}

// PhiT_J[j][l] = X_J[l][j] in the storage precision; optionally also the dense Phi
// (n x n0, FP64) with the interface indicator.
template <typename TP>
__global__ void k_store_phiT(const double* __restrict__ X, const int64_t* __restrict__ toff,
                             const int32_t* __restrict__ ldt, const int32_t* __restrict__ part_of_row,
                             const int64_t* __restrict__ ioff, int64_t nrows, const int64_t* __restrict__ coff,
                             const int64_t* __restrict__ phioff, const int32_t* __restrict__ phild, TP* __restrict__ phiT,
                             const int32_t* __restrict__ idofs, const int32_t* __restrict__ cols, double* __restrict__ dense,
                             int64_t n0) {
  int64_t row = blockIdx.x;
  if (row >= nrows) return;
  int J = part_of_row[row];
  int64_t l = row - ioff[J];
  int c = int(coff[J + 1] - coff[J]);
  const double* x = X + toff[J] + l * ldt[J];
  for (int j = threadIdx.x; j < c; j += blockDim.x) {
    phiT[phioff[J] + int64_t(j) * phild[J] + l] = TP(x[j]);
    if (dense) dense[int64_t(idofs[row]) * n0 + cols[coff[J] + j]] = x[j];
  }
}

template <typename TP>
void store_phiT(const double* X, const int64_t* toff, const int32_t* ldt, const int32_t* part_of_row,
                const int64_t* ioff, int64_t nrows, const int64_t* coff, const int64_t* phioff, const int32_t* phild,
                TP* phiT, const int32_t* idofs, const int32_t* cols, double* dense, int64_t n0, cudaStream_t s) {
  if (nrows == 0) return;
  k_store_phiT<TP><<<int(nrows), 128, 0, s>>>(X, toff, ldt, part_of_row, ioff, nrows, coff, phioff, phild, phiT, idofs,
                                              cols, dense, n0);
  check_launch("k_store_phiT");
}
template void store_phiT<double>(const double*, const int64_t*, const int32_t*, const int32_t*, const int64_t*,
                                 int64_t, const int64_t*, const int64_t*, const int32_t*, double*, const int32_t*,
                                 const int32_t*, double*, int64_t, cudaStream_t);
template void store_phiT<float>(const double*, const int64_t*, const int32_t*, const int32_t*, const int64_t*, int64_t,
                                const int64_t*, const int64_t*, const int32_t*, float*, const int32_t*, const int32_t*,
                                double*, int64_t, cudaStream_t);

__global__ void k_dense_gamma(const int32_t* __restrict__ gdofs, const int32_t* __restrict__ gcol, int64_t ng,
                              double* __restrict__ dense, int64_t n0) {
  int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q < ng) dense[int64_t(gdofs[q]) * n0 + gcol[q]] = 1.0;
}
void dense_gamma(const int32_t* gdofs, const int32_t* gcol, int64_t ng, double* dense, int64_t n0, cudaStream_t s) {
  if (ng == 0) return;
  k_dense_gamma<<<int((ng + 255) / 256), 256, 0, s>>>(gdofs, gcol, ng, dense, n0);
  check_launch("k_dense_gamma");
}

}  // namespace gdsw

namespace gdsw {
void launch_tneg(const MatView& A, const SlabView& S, const int32_t* gamma_ptr, const int32_t* gcol,
                 const double* gval, const int32_t* cols,
                 const int64_t* coff, const int64_t* toff, const int32_t* ldt, double* T, int* err, cudaStream_t s) {
  if (S.nvec == 0) return;
  k_tneg<<<int((S.nvec + 127) / 128), 128, 0, s>>>(A, S, gamma_ptr, gcol, gval, cols, coff, toff, ldt, T, err);
  check_launch("k_tneg");
}
void launch_yint(const MatView& A, const SlabView& S, const int32_t* ilocal, const int64_t* coff, const int64_t* toff,
                 const int32_t* ldt, const double* X, const double* Tn, double* Y, cudaStream_t s) {
  if (S.nvec == 0) return;
  k_yint<<<int((S.nvec + 7) / 8), 256, 0, s>>>(A, S, ilocal, coff, toff, ldt, X, Tn, Y);
  check_launch("k_yint");
}
}  // namespace gdsw
