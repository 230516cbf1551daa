// Overlapping Schwarz data movement and the GDSW coarse transfer, on every level
// (arXiv 2606.01433, Section 2.1: R_i r, sum_i R_i^T (.) and Phi^T r / Phi x; Section 2.2:
// the same on the coarse decompositions).  Every reduction has a fixed order, so results
// are bitwise reproducible run to run.
#include "common.h"
#include "kernels.h"

namespace gdsw {

// r_i = R_i r for all parts at once: one thread per local position, cast to the local
// precision on the fly.
template <typename TV>
__global__ void k_gather(const double* __restrict__ r, const int32_t* __restrict__ idx, TV* __restrict__ out,
                         int64_t n) {
  dep_release();
  dep_wait();
  int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p < n) out[p] = TV(r[__ldg(idx + p)]);
}

template <typename TV>
void launch_gather(const double* r, const int32_t* idx, TV* out, int64_t n, cudaStream_t s) {
  if (n == 0) return;
  launch_chained(k_gather<TV>, dim3(unsigned((n + 255) / 256)), dim3(256), 0, s, r, idx, out, n);
  check_launch("k_gather");
}
template void launch_gather<double>(const double*, const int32_t*, double*, int64_t, cudaStream_t);
template void launch_gather<float>(const double*, const int32_t*, float*, int64_t, cudaStream_t);

// z[g] = sum over the overlapping copies of dof g of w * x_i[local] (partition-of-unity
// weights, or 1 for the plain sum), accumulated in FP64 in list order.
template <typename TV>
__global__ void k_scatter(const TV* __restrict__ x, const int32_t* __restrict__ ptr, const int32_t* __restrict__ pos,
                          const double* __restrict__ w, double* __restrict__ z, int n, int accumulate) {
  dep_release();
  dep_wait();
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  double acc = 0.0;
  for (int e = ptr[g]; e < ptr[g + 1]; ++e) acc = fma(w[e], double(x[pos[e]]), acc);
  z[g] = accumulate ? z[g] + acc : acc;
}

template <typename TV>
void launch_scatter(const TV* x, const int32_t* ptr, const int32_t* pos, const double* w, double* z, int n,
                    int accumulate, cudaStream_t s) {
  if (n == 0) return;
  launch_chained(k_scatter<TV>, dim3(unsigned((n + 255) / 256)), dim3(256), 0, s, x, ptr, pos, w, z, n, accumulate);
  check_launch("k_scatter");
}
template void launch_scatter<double>(const double*, const int32_t*, const int32_t*, const double*, double*, int, int,
                                     cudaStream_t);
template void launch_scatter<float>(const float*, const int32_t*, const int32_t*, const double*, double*, int, int,
                                    cudaStream_t);

// Restriction r0 = Phi^T r in two deterministic passes over the stored Phi_I^T blocks.
// Pass 1 (k_restrict_tiles): one CTA per 256-dof tile of a part's interior (the prolongation's
// tiles); the tile's residual entries are gathered once into shared memory (in the basis
// precision).  Warp w takes rows j = w + 8 i of PhiT_J, four rows per step, each lane reading
// one 16-byte vector per row per 32 V columns, so a step has eight (FP32) or sixteen (FP64)
// 16-byte loads in flight per lane and the basis is read exactly once.  Lane sums (basis
// precision) go to shared memory, [row][lane] with rows padded to 33; after the tile, one
// thread per row adds its 32 lane sums in FP64 in lane order and stores the tile's partial.
// Pass 2 (k_restrict_reduce): one warp per coarse column k adds, for each (part, row) that
// carries k, that row's tile partials in tile order, then the Phi_Gamma entries of k.
template <typename TP>
struct ProAcc {
  using X = double;
};
template <>
struct ProAcc<float> {
  using X = float;
};

template <typename TP>
__global__ void __launch_bounds__(256) k_restrict_tiles(const TP* __restrict__ phiT, const ProMeta* __restrict__ meta,
                                                        const int32_t* __restrict__ tile_part,
                                                        const int32_t* __restrict__ tile_col0,
                                                        const int32_t* __restrict__ tile_rank,
                                                        const int64_t* __restrict__ part_poff,
                                                        const int32_t* __restrict__ part_ntiles,
                                                        const int32_t* __restrict__ idofs,
                                                        const double* __restrict__ r, double* __restrict__ partial) {
  using X = typename ProAcc<TP>::X;
  constexpr int V = 16 / sizeof(TP), NC = 256 / (32 * V);  // elements per 16-byte load; loads per lane per row
  extern __shared__ __align__(16) unsigned char rt_smem[];
  X* rs = reinterpret_cast<X*>(rt_smem);                      // 256 residual entries
  X* lsum = rs + 256;                                          // [row][lane] lane sums, rows of 33
  dep_release();  // launched in plain stream order (it follows a wait on the main stream)
  const int J = tile_part[blockIdx.x];
  const ProMeta m = meta[J];
  const int col0 = tile_col0[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int span = min(256, m.ld - col0);   // stored row length left in this tile (a multiple of 8)
  // rows j0, j0 + 8, j0 + 16, j0 + 24 of the tile, one 16-byte vector per lane and 32 V columns
  auto load_step = [&](int j0, uint4 (&v)[4][NC]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + 8 * q;
      const TP* row = phiT + m.phi + int64_t(j) * m.ld + col0;
#pragma unroll
      for (int u = 0; u < NC; ++u) {
        const int t = (lane + 32 * u) * V;
        v[q][u] = (j < m.c && t < span) ? __ldcs(reinterpret_cast<const uint4*>(row + t)) : make_uint4(0, 0, 0, 0);
      }
    }
  };
  auto use_step = [&](int j0, const uint4 (&v)[4][NC]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + 8 * q;
      X acc = X(0);
#pragma unroll
      for (int u = 0; u < NC; ++u) {
        const TP* e = reinterpret_cast<const TP*>(&v[q][u]);
#pragma unroll
        for (int k = 0; k < V; ++k) acc = fma(X(e[k]), rs[(lane + 32 * u) * V + k], acc);
      }
      if (j < m.c) lsum[j * 33 + lane] = acc;
    }
  };
  // the first step's basis loads go out before the residual gather and its barrier
  uint4 va[4][NC];
  load_step(warp, va);
  const int l = col0 + int(threadIdx.x);
  rs[threadIdx.x] = l < m.nI ? X(r[idofs[m.ioff + l]]) : X(0);
  __syncthreads();
  for (int j0 = warp; j0 < m.c; j0 += 32) {
    if (j0 > warp) load_step(j0, va);
    use_step(j0, va);
  }
  __syncthreads();
  const int64_t pbase = part_poff[J] + tile_rank[blockIdx.x];
  const int nt = part_ntiles[J];
  for (int j = threadIdx.x; j < m.c; j += blockDim.x) {
    double s = 0.0;
#pragma unroll 8
    for (int q = 0; q < 32; ++q) s += double(lsum[j * 33 + q]);
    partial[pbase + int64_t(j) * nt] = s;
  }
}

// r0[k] = sum over the (part, row) entries q of column k of the row's tile partials
// (partial[q_start[q] .. + q_count[q]], in tile order) + sum of the Phi_Gamma entries of k
// times r.  One warp per coarse dof; lane-strided partial sums and a fixed butterfly.
__global__ void k_restrict_reduce(const double* __restrict__ partial, const int64_t* __restrict__ q_start,
                                  const int32_t* __restrict__ q_count, const double* __restrict__ r,
                                  const int32_t* __restrict__ rr_ptr, const int32_t* __restrict__ rr_pos,
                                  const int32_t* __restrict__ rg_ptr, const int32_t* __restrict__ rg_dof,
                                  const double* __restrict__ rg_val, double* __restrict__ r0, int n0) {
  dep_release();
  dep_wait();
  int k = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (k >= n0) return;
  double acc = 0.0;
  for (int e = rr_ptr[k] + lane; e < rr_ptr[k + 1]; e += 32) {
    const int q = rr_pos[e];
    const double* p = partial + q_start[q];
    double t = 0.0;
    for (int i = 0; i < q_count[q]; ++i) t += p[i];
    acc += t;
  }
  for (int e = rg_ptr[k] + lane; e < rg_ptr[k + 1]; e += 32) acc = fma(rg_val[e], r[rg_dof[e]], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) r0[k] = acc;
}

void launch_restrict(const LevelDev& L, const double* r, double* r0, cudaStream_t s) {
  if (L.n0 == 0) return;
  const ProMeta* meta = reinterpret_cast<const ProMeta*>(L.pro_meta);
  if (L.n_pro_tiles > 0) {
    const size_t es = L.phi_prec == GDSW_FP64 ? 8 : 4;
    const size_t smem = es * (256 + 33 * size_t(L.max_c));
    if (L.phi_prec == GDSW_FP64)
      k_restrict_tiles<double><<<L.n_pro_tiles, 256, smem, s>>>(static_cast<const double*>(L.phiT), meta,
                                                                L.pro_tile_part, L.pro_tile_col0, L.pro_tile_rank,
                                                                L.part_poff, L.part_ntiles, L.idofs, r, L.partial);
    else
      k_restrict_tiles<float><<<L.n_pro_tiles, 256, smem, s>>>(static_cast<const float*>(L.phiT), meta,
                                                               L.pro_tile_part, L.pro_tile_col0, L.pro_tile_rank,
                                                               L.part_poff, L.part_ntiles, L.idofs, r, L.partial);
    check_launch("k_restrict_tiles");
  }
  launch_chained(k_restrict_reduce, dim3(unsigned((L.n0 + 7) / 8)), dim3(256), 0, s, L.partial, L.q_start,
                 L.q_count, r, L.rr_ptr, L.rr_pos, L.rg_ptr, L.rg_dof, L.rg_val, r0, L.n0);
  check_launch("k_restrict_reduce");
}

// z[I_J[l]] += sum_j PhiT_J[j][l] x0[cols_J[j]]: one thread per interior dof, coalesced
// along the rows of the stored transpose; every interior dof belongs to exactly one part.
// Accumulation precision follows the stored basis: an FP64 basis accumulates in FP64; an FP32
// basis forms each run of eight products in FP32 (x0 rounded to FP32 in shared memory, the
// precision the basis itself carries) and adds the run totals in FP64, so the kernel issues
// one FP64 add per eight columns instead of one FP64 FMA per column -- GB300's FP64 pipe
// would otherwise bound it, far below the memory rate.
template <typename TP>
__global__ void __launch_bounds__(256) k_prolong(const TP* __restrict__ phiT, const ProMeta* __restrict__ meta,
                                                 const int32_t* __restrict__ tile_part,
                                                 const int32_t* __restrict__ tile_col0,
                                                 const int32_t* __restrict__ idofs, const int32_t* __restrict__ cols,
                                                 const double* __restrict__ x0, double* __restrict__ z) {
  using X = typename ProAcc<TP>::X;
  extern __shared__ double xs_raw[];
  X* xs = reinterpret_cast<X*>(xs_raw);
  dep_release();  // launched in plain stream order (it follows a wait on the coarse stream)
  const int J = tile_part[blockIdx.x];
  const ProMeta m = meta[J];
  for (int j = threadIdx.x; j < m.c; j += blockDim.x) xs[j] = X(x0[cols[m.coff + j]]);
  __syncthreads();
  const int l = tile_col0[blockIdx.x] + threadIdx.x;
  if (l >= m.nI) return;
  double acc = 0.0;
  const TP* p = phiT + m.phi + l;
  int j = 0;
  for (; j + 16 <= m.c; j += 16) {  // sixteen independent loads in flight, products in column order
    TP v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = __ldcs(p + int64_t(j + u) * m.ld);
#pragma unroll
    for (int h = 0; h < 16; h += 8) {
      X part = X(0);
#pragma unroll
      for (int u = 0; u < 8; ++u) part = fma(X(v[h + u]), xs[j + h + u], part);
      acc += double(part);
    }
  }
  for (; j + 8 <= m.c; j += 8) {
    TP v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcs(p + int64_t(j + u) * m.ld);
    X part = X(0);
#pragma unroll
    for (int u = 0; u < 8; ++u) part = fma(X(v[u]), xs[j + u], part);
    acc += double(part);
  }
  X part = X(0);
  for (; j < m.c; ++j) part = fma(X(__ldcs(p + int64_t(j) * m.ld)), xs[j], part);
  acc += double(part);
  int64_t g = idofs[m.ioff + l];
  z[g] += acc;
}

// z[g] += sum over the Phi_Gamma entries of interface dof g of value * x0[column], one thread
// per interface dof, entries in column order
__global__ void k_axpy_gamma(const int32_t* __restrict__ gu_dof, const int32_t* __restrict__ gu_ptr,
                             const int32_t* __restrict__ gcol, const double* __restrict__ gval, int64_t ngu,
                             const double* __restrict__ x0, double* __restrict__ z) {
  dep_release();
  dep_wait();
  int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= ngu) return;
  double acc = 0.0;
  for (int32_t e = gu_ptr[q]; e < gu_ptr[q + 1]; ++e) acc = fma(gval[e], x0[gcol[e]], acc);
  z[gu_dof[q]] += acc;
}

void launch_prolong(const LevelDev& L, const double* x0, double* z, cudaStream_t s) {
  if (L.n0 == 0) return;
  if (L.n_pro_tiles > 0) {
    size_t smem = size_t(L.max_c) * sizeof(double);
    const ProMeta* meta = reinterpret_cast<const ProMeta*>(L.pro_meta);
    if (L.phi_prec == GDSW_FP64)
      k_prolong<double><<<L.n_pro_tiles, 256, smem, s>>>(static_cast<const double*>(L.phiT), meta, L.pro_tile_part,
                                                         L.pro_tile_col0, L.idofs, L.cols, x0, z);
    else
      k_prolong<float><<<L.n_pro_tiles, 256, smem, s>>>(static_cast<const float*>(L.phiT), meta, L.pro_tile_part,
                                                        L.pro_tile_col0, L.idofs, L.cols, x0, z);
    check_launch("k_prolong");
  }
}

void launch_axpy_gamma(const int32_t* gu_dof, const int32_t* gu_ptr, const int32_t* gcol, const double* gval,
                       int64_t ngu, const double* x0, double* z, cudaStream_t s) {
  if (ngu == 0) return;
  launch_chained(k_axpy_gamma, dim3(unsigned((ngu + 255) / 256)), dim3(256), 0, s, gu_dof, gu_ptr, gcol, gval, ngu,
                 x0, z);
  check_launch("k_axpy_gamma");
}

void set_prolong_smem_limits() {
  cudaFuncSetAttribute(k_prolong<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_prolong<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_restrict_tiles<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_restrict_tiles<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace gdsw
