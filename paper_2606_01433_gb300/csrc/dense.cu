// Batched dense kernels: the ragged GEMV that carries every local and coarse solve of the
// preconditioner apply (arXiv 2606.01433, Section 2.1/2.2: the A_i^{-1} terms, applied as
// block-LDU sweeps with explicit inverse diagonal blocks), and the set-up kernels that
// build those factors: a batched GEMM and a batched blocked Gauss-Jordan inverse with
// partial pivoting.
#include <cfloat>

#include "common.h"
#include "kernels.h"

namespace gdsw {

// ------------------------------------------------------------------ load helpers
template <typename T> struct Vec16;
template <> struct Vec16<double> { static constexpr int N = 2; };
template <> struct Vec16<float> { static constexpr int N = 4; };
template <> struct Vec16<__nv_bfloat16> { static constexpr int N = 8; };

__device__ __forceinline__ void load16(const double* p, double* v) {
  double2 t = __ldg(reinterpret_cast<const double2*>(p));
  v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void load16(const float* p, float* v) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load16(const __nv_bfloat16* p, float* v) {
  uint4 t = __ldg(reinterpret_cast<const uint4*>(p));
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&t);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float2 f = __bfloat1622float2(h[q]);
    v[2 * q] = f.x; v[2 * q + 1] = f.y;
  }
}
// streaming (evict-first) variant for matrices read once per apply
__device__ __forceinline__ void load16s(const double* p, double* v) {
  double2 t = __ldcs(reinterpret_cast<const double2*>(p));
  v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void load16s(const float* p, float* v) {
  float4 t = __ldcs(reinterpret_cast<const float4*>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load16s(const __nv_bfloat16* p, float* v) {
  uint4 t = __ldcs(reinterpret_cast<const uint4*>(p));
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&t);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float2 f = __bfloat1622float2(h[q]);
    v[2 * q] = f.x; v[2 * q + 1] = f.y;
  }
}

// ------------------------------------------------------------------ overlapped launch chain
// The local sweeps are chains of launches: each slab step reads the vectors the previous one
// wrote.  Each launch of the chain is a programmatic dependent launch (common.h): its CTAs may
// become resident while the previous launch drains its last wave, prefetch the start of their
// factor rows into L2 (the factors do not depend on the previous launch), and wait for the
// previous grid before reading a vector.
bool g_launch_overlap = true;

// raw 16-byte streaming load, unpacked only at the multiply (keeps BF16 tiles at half the
// registers of unpacked floats)
__device__ __forceinline__ uint4 ldraw(const void* p) { return __ldcs(reinterpret_cast<const uint4*>(p)); }
template <typename TM> struct Unpack;
template <> struct Unpack<double> {
  static __device__ __forceinline__ void run(const uint4& r, double* v) {
    v[0] = __hiloint2double(int(r.y), int(r.x));
    v[1] = __hiloint2double(int(r.w), int(r.z));
  }
};
template <> struct Unpack<float> {
  static __device__ __forceinline__ void run(const uint4& r, float* v) {
    v[0] = __uint_as_float(r.x); v[1] = __uint_as_float(r.y); v[2] = __uint_as_float(r.z); v[3] = __uint_as_float(r.w);
  }
};
template <> struct Unpack<__nv_bfloat16> {
  static __device__ __forceinline__ void run(const uint4& r, float* v) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&r);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2 f = __bfloat1622float2(h[q]);
      v[2 * q] = f.x; v[2 * q + 1] = f.y;
    }
  }
};

// ------------------------------------------------------------------ ragged batched GEMV
// One CTA = 8 warps = ROWS rows of one task; each warp owns ROWS/8 rows and streams them
// with 16-byte loads (four rows in flight per warp).  The task's input vector is staged in
// shared memory once per CTA.  y[r] = base[r] + alpha * sum_c M[r][c] x[c].
// Symmetric block stored as its upper-triangle tiles (T x T, T = 32 lanes x one 16-byte load,
// tiles (I, J >= I) in row-major order, zero padded): one CTA reads tile (I, J) once and
// produces both S_IJ x_J (rows of block I) and, off the diagonal, S_IJ^T x_I (rows of block
// J) as partial sums; k_sym_reduce adds the partials of each row in a fixed order.
template <typename TM, typename TV>
__device__ __forceinline__ void sym_tile(const TM* __restrict__ M, const TV* xbase, TV* part, const GemvTask& t,
                                         int I, int J, TV* smem) {
  constexpr int V = Vec16<TM>::N, T = 32 * V, RW = T / 8;
  TV* xi = smem;
  TV* xj = smem + T;
  TV* prow = smem + 2 * T;
  TV* pcol = smem + 3 * T;  // 8 x T
  const int s = t.rows, nt = t.ld;
  for (int e = threadIdx.x; e < T; e += blockDim.x) {
    xi[e] = I * T + e < s ? __ldcg(xbase + t.x + I * T + e) : TV(0);
    xj[e] = J * T + e < s ? __ldcg(xbase + t.x + J * T + e) : TV(0);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tidx = int64_t(I) * nt - int64_t(I) * (I - 1) / 2 + (J - I);
  const TM* tp = M + t.mat + tidx * T * T + int64_t(warp * RW) * T + lane * V;
  TV colacc[V], rowacc[RW];
#pragma unroll
  for (int u = 0; u < V; ++u) colacc[u] = TV(0);
#pragma unroll
  for (int rr = 0; rr < RW; rr += 4) {
    TV v[4][V];
#pragma unroll
    for (int q = 0; q < 4; ++q) load16s(tp + int64_t(rr + q) * T, v[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const TV xr = xi[warp * RW + rr + q];
      TV d = TV(0);
#pragma unroll
      for (int u = 0; u < V; ++u) {
        d = fma(v[q][u], xj[lane * V + u], d);
        colacc[u] = fma(v[q][u], xr, colacc[u]);
      }
      rowacc[rr + q] = d;
    }
  }
#pragma unroll
  for (int rr = 0; rr < RW; ++rr) {
    TV d = rowacc[rr];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) prow[warp * RW + rr] = d;
  }
#pragma unroll
  for (int u = 0; u < V; ++u) pcol[warp * T + lane * V + u] = colacc[u];
  __syncthreads();
  for (int e = threadIdx.x; e < T; e += blockDim.x) {
    part[t.part + (int64_t(I) * nt + J) * T + e] = prow[e];
    if (I != J) {
      TV cs = pcol[e];
#pragma unroll
      for (int w = 1; w < 8; ++w) cs += pcol[w * T + e];
      part[t.part + (int64_t(J) * nt + I) * T + e] = cs;
    }
  }
}

// Rows [row0, row0 + 8 RPW G) of one task: G consecutive groups of 8 RPW rows share one
// staging of the input vector, and every row is one warp's dot product in the same order
// whatever G is.  Vector reads go through L2 (ld.global.cg): in the persistent sweep other
// CTAs write the local vectors while this one runs.
template <typename TM, typename TV, int RPW, int G>
__device__ __forceinline__ void rows_tile(const TM* __restrict__ M, const TV* xbase, TV* ybase, const TV* bbase,
                                          const GemvTask& t, int row0, TV* xs) {
  const int ld = t.ld;
  for (int c = threadIdx.x; c < ld; c += blockDim.x) xs[c] = c < t.cols ? __ldcg(xbase + t.x + c) : TV(0);
  __syncthreads();
  constexpr int V = Vec16<TM>::N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int g = 0; g < G; ++g) {  // G is a compile-time constant: a runtime count here slows the loads
    const int rbeg = row0 + g * 8 * RPW + warp * RPW;
    if (rbeg - warp * RPW >= t.rows) break;
    TV acc[RPW];
    const TM* rowp[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      acc[q] = TV(0);
      int r = rbeg + q;
      rowp[q] = M + t.mat + int64_t(r < t.rows ? r : 0) * ld;
    }
    int c = lane * V;
    for (; c + 32 * V < ld; c += 64 * V) {  // two column chunks per row in flight
      uint4 m0[RPW], m1[RPW];
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        if (rbeg + q < t.rows) {
          m0[q] = ldraw(rowp[q] + c);
          m1[q] = ldraw(rowp[q] + c + 32 * V);
        }
      }
      TV xv0[V], xv1[V];
#pragma unroll
      for (int u = 0; u < V; ++u) {
        xv0[u] = xs[c + u];
        xv1[u] = xs[c + 32 * V + u];
      }
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        if (rbeg + q < t.rows) {
          TV mv0[V], mv1[V];
          Unpack<TM>::run(m0[q], mv0);
          Unpack<TM>::run(m1[q], mv1);
#pragma unroll
          for (int u = 0; u < V; ++u) acc[q] = fma(mv1[u], xv1[u], fma(mv0[u], xv0[u], acc[q]));
        }
      }
    }
    if (c < ld) {
      TV xv[V];
#pragma unroll
      for (int u = 0; u < V; ++u) xv[u] = xs[c + u];
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        if (rbeg + q < t.rows) {
          TV mv[V];
          load16s(rowp[q] + c, mv);
#pragma unroll
          for (int u = 0; u < V; ++u) acc[q] = fma(mv[u], xv[u], acc[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    }
    if (lane < RPW) {
      TV a = acc[0];
#pragma unroll
      for (int q = 1; q < RPW; ++q)
        if (lane == q) a = acc[q];
      int r = rbeg + lane;
      if (r < t.rows) {
        TV v = TV(t.alpha) * a;
        if (t.base >= 0) v += __ldcg(bbase + t.base + r);
        ybase[t.y + r] = v;
      }
    }
  }
}

template <typename TM, typename TV, int RPW, int G>
__global__ void __launch_bounds__(256) k_gemv(const TM* __restrict__ M, const TV* xbase, TV* ybase,
                                              const TV* bbase, const GemvTask* __restrict__ tasks,
                                              const GemvTile* __restrict__ tiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TV* xs = reinterpret_cast<TV*>(smem_raw);
  const GemvTile tl = tiles[blockIdx.x];
  const GemvTask t = tasks[tl.task];
  dep_release();
  {  // factor prefetch before the dependency wait: the first 2 KB of the warp's first rows, or
     // the first eight rows of the warp's part of a symmetric tile
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (t.kind == 1) {
      constexpr int T = 32 * Vec16<TM>::N, RW = T / 8;
      const int I = tl.row0 >> 16, J = tl.row0 & 0xffff;
      const int64_t tidx = int64_t(I) * t.ld - int64_t(I) * (I - 1) / 2 + (J - I);
      prefetch_l2(M + t.mat + tidx * T * T + int64_t(warp * RW + (lane >> 2)) * T + (lane & 3) * (128 / sizeof(TM)));
    } else {
      for (int q = lane >> 4; q < RPW; q += 2) {
        const int r = tl.row0 + warp * RPW + q;
        const int off = (lane & 15) * int(128 / sizeof(TM));
        if (r < t.rows && off < t.ld) prefetch_l2(M + t.mat + int64_t(r) * t.ld + off);
      }
    }
  }
  dep_wait();
  if (t.kind == 1)  // packed symmetric tile; partial sums go to ybase + t.part
    sym_tile<TM, TV>(M, xbase, ybase, t, tl.row0 >> 16, tl.row0 & 0xffff, xs);
  else
    rows_tile<TM, TV, RPW, G>(M, xbase, ybase, bbase, t, tl.row0, xs);
}

// ------------------------------------------------------------------ ragged batched GEMV, transposed
// y[c] = base[c] + alpha * sum_r M[r][c] x[r] for the columns [col0, col0 + LW V) of a task
// (used with the sub-diagonal blocks G of a symmetric LDL^T factorisation, whose
// transposes are the super-diagonal blocks).  A group of LW lanes reads one row of the tile
// (a lane owns V consecutive columns, one 16-byte load); the 256 / LW groups split the rows,
// four rows in flight each; the partial sums of a column are combined in shared memory in a
// fixed order.  Narrow tiles (LW V columns) give many CTAs per task, so the ragged launch
// (tasks of different heights) spreads evenly over the SMs.
// lanes per tile row of the transposed GEMV: half warps
template <typename TM> struct ColsLanes { static constexpr int LW = 16; };

template <typename TM, typename TV>
__device__ __forceinline__ void cols_tile(const TM* __restrict__ M, const TV* xbase, TV* ybase, const TV* bbase,
                                          const GemvTask& t, int col0, TV* xs, TV* part) {
  constexpr int V = Vec16<TM>::N, LW = ColsLanes<TM>::LW, C = LW * V, NG = 256 / LW;
  for (int r = threadIdx.x; r < t.rows; r += blockDim.x) xs[r] = __ldcg(xbase + t.x + r);
  __syncthreads();
  const int ll = threadIdx.x % LW, grp = threadIdx.x / LW;  // NG row groups of LW lanes
  const int c0 = col0 + ll * V;  // tile column start + this lane's V columns
  TV acc[V];
#pragma unroll
  for (int u = 0; u < V; ++u) acc[u] = TV(0);
  if (c0 < t.ld) {
    const TM* p = M + t.mat + c0;
    int r = grp;
    for (; r + 3 * NG < t.rows; r += 4 * NG) {
      TV v[4][V];
#pragma unroll
      for (int q = 0; q < 4; ++q) load16s(p + int64_t(r + NG * q) * t.ld, v[q]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const TV xq = xs[r + NG * q];
#pragma unroll
        for (int u = 0; u < V; ++u) acc[u] = fma(v[q][u], xq, acc[u]);
      }
    }
    for (; r < t.rows; r += NG) {
      TV v0[V];
      load16s(p + int64_t(r) * t.ld, v0);
      const TV x0 = xs[r];
#pragma unroll
      for (int u = 0; u < V; ++u) acc[u] = fma(v0[u], x0, acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < V; ++u) part[grp * (C + 1) + ll * V + u] = acc[u];
  __syncthreads();
  for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
    const int c = col0 + cc;
    if (c < t.cols) {
      TV s = part[cc];
#pragma unroll
      for (int g = 1; g < NG; ++g) s += part[g * (C + 1) + cc];
      TV v = TV(t.alpha) * s;
      if (t.base >= 0) v += __ldcg(bbase + t.base + c);
      ybase[t.y + c] = v;
    }
  }
}

template <typename TM, typename TV>
__global__ void __launch_bounds__(256) k_gemvt(const TM* __restrict__ M, const TV* xbase, TV* ybase,
                                               const TV* bbase, const GemvTask* __restrict__ tasks,
                                               const GemvTile* __restrict__ tiles) {
  constexpr int LW = ColsLanes<TM>::LW, C = LW * Vec16<TM>::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ TV part[(256 / LW) * (C + 1)];
  const GemvTile tl = tiles[blockIdx.x];
  const GemvTask t = tasks[tl.task];
  dep_release();
  {  // factor prefetch before the dependency wait: the tile's first 128 rows (two lines each)
    const int r = threadIdx.x >> 1, off = tl.row0 + (threadIdx.x & 1) * int(128 / sizeof(TM));
    if (r < t.rows && off < t.ld) prefetch_l2(M + t.mat + int64_t(r) * t.ld + off);
  }
  dep_wait();
  cols_tile<TM, TV>(M, xbase, ybase, bbase, t, tl.row0, reinterpret_cast<TV*>(smem_raw), part);
}

template <typename TM, typename TV>
void launch_gemv(const TM* M, const TV* x, TV* y, const TV* b, const GemvPlan& P, int launch, int max_ld,
                 cudaStream_t s) {
  int t0 = P.launch_tile_off[launch], t1 = P.launch_tile_off[launch + 1];
  if (t1 <= t0) return;
  size_t smem = size_t(max_ld) * sizeof(TV);
  const unsigned nb = unsigned(t1 - t0);
  const GemvTile* tl = P.d_tiles + t0;
  if (P.transposed) {
    launch_chained(k_gemvt<TM, TV>, dim3(nb), dim3(256), smem, s, M, x, y, b, P.d_tasks, tl);
    check_launch("k_gemvt");
  } else {
    if (P.rows_per_tile == 128)
      launch_chained(k_gemv<TM, TV, 4, 4>, dim3(nb), dim3(256), smem, s, M, x, y, b, P.d_tasks, tl);
    else if (P.rows_per_tile == 64)
      launch_chained(k_gemv<TM, TV, 4, 2>, dim3(nb), dim3(256), smem, s, M, x, y, b, P.d_tasks, tl);
    else
      launch_chained(k_gemv<TM, TV, 4, 1>, dim3(nb), dim3(256), smem, s, M, x, y, b, P.d_tasks, tl);
    check_launch("k_gemv");
  }
}

// y[r] = alpha * sum over the nt source blocks of the partials of row r (fixed order);
// one CTA per 256 rows of one symmetric task.
template <typename TV>
__device__ __forceinline__ void reduce_tile(const TV* vec, TV* ybase, const GemvTask& t, int row0, int T) {
  const int r = row0 + threadIdx.x;
  if (r >= t.rows) return;
  const int R = r / T, e = r - R * T;
  const TV* p = vec + t.part + int64_t(R) * t.ld * T + e;
  TV s = TV(0);
  for (int S = 0; S < t.ld; ++S) s += __ldcg(p + int64_t(S) * T);
  ybase[t.y + r] = TV(t.alpha) * s;
}

template <typename TV>
__global__ void k_sym_reduce(const TV* __restrict__ vec, TV* ybase, const GemvTask* __restrict__ tasks,
                             const GemvTile* __restrict__ tiles, int T) {
  const GemvTile tl = tiles[blockIdx.x];
  const GemvTask t = tasks[tl.task];
  dep_release();
  dep_wait();
  reduce_tile<TV>(vec, ybase, t, tl.row0, T);
}

template <typename TV>
void launch_sym_reduce(const TV* vec, TV* y, const GemvPlan& P, int T, cudaStream_t s) {
  int t0 = P.launch_tile_off[0], t1 = P.launch_tile_off[1];
  if (t1 <= t0) return;
  launch_chained(k_sym_reduce<TV>, dim3(unsigned(t1 - t0)), dim3(256), 0, s, vec, y, P.d_tasks, P.d_tiles + t0, T);
  check_launch("k_sym_reduce");
}
template void launch_sym_reduce<double>(const double*, double*, const GemvPlan&, int, cudaStream_t);
template void launch_sym_reduce<float>(const float*, float*, const GemvPlan&, int, cudaStream_t);

// ------------------------------------------------------------------ persistent level sweep
// One launch runs every tile of a level's local solves -- forward row tiles and packed
// symmetric tiles, the partial-sum reductions, the transposed backward tiles -- from a work
// list in dependency order.  CTAs claim items with an atomic counter (the next claim is made
// before the current item runs).  An item first waits until the per-slab counters of the
// tiles it reads from are complete (y_k written, partials written, w_k written, x_k
// written), runs, then adds one to its own counter.  Claims follow list order and every
// producer precedes its consumers in the list, so the lowest unfinished claimed item always
// has its producers finished: the sweep cannot deadlock, whatever the number of resident
// CTAs.  A wait longer than limit_ns sets *flag and every CTA returns; the host reports it.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool wait_count(const unsigned* cnt, unsigned need, unsigned* flag,
                                           unsigned long long limit_ns) {
  const volatile unsigned* c = cnt;
  if (*c >= need) return true;
  const unsigned long long t_end = global_ns() + limit_ns;
  while (*c < need) {
    if (*reinterpret_cast<volatile unsigned*>(flag)) return false;
    if (global_ns() > t_end) {
      atomicExch(flag, 1u);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

template <typename TM, typename TV, int G>
__global__ void __launch_bounds__(256, 3) k_sweep(const TM* __restrict__ M, TV* vec, const GemvTask* __restrict__ tasks,
                                               const SweepItem* __restrict__ items, int nitems, unsigned* ctr,
                                               unsigned* flag, int T, int xs_elems, unsigned long long limit_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TV* xs = reinterpret_cast<TV*>(smem_raw);
  TV* cpart = xs + xs_elems;  // column partials of the transposed tiles
  __shared__ int s_item[2];
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_item[0] = int(atomicAdd(ctr, 1u));
  __syncthreads();
  int cur = 0;
  while (true) {
    const int it = s_item[cur];
    if (it >= nitems) break;
    const SweepItem w = items[it];
    if (threadIdx.x == 0) {
      s_item[cur ^ 1] = int(atomicAdd(ctr, 1u));
      bool ok = true;
      if (w.wait0 >= 0) ok = wait_count(ctr + w.wait0, unsigned(w.need0), flag, limit_ns);
      if (ok && w.wait1 >= 0) ok = wait_count(ctr + w.wait1, unsigned(w.need1), flag, limit_ns);
      __threadfence();
      s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) break;
    const GemvTask t = tasks[w.task];
    if (w.op == SWEEP_ROWS)
      rows_tile<TM, TV, 4, G>(M, vec, vec, vec, t, w.arg, xs);
    else if (w.op == SWEEP_SYM)
      sym_tile<TM, TV>(M, vec, vec, t, w.arg >> 16, w.arg & 0xffff, xs);
    else if (w.op == SWEEP_REDUCE)
      reduce_tile<TV>(vec, vec, t, w.arg, T);
    else
      cols_tile<TM, TV>(M, vec, vec, vec, t, w.arg, xs, cpart);
    __syncthreads();  // every write of this item is issued; the shared staging is free again
    if (threadIdx.x == 0 && w.signal >= 0) {
      __threadfence();
      atomicAdd(ctr + w.signal, 1u);
    }
    cur ^= 1;
  }
}

template <typename TM, typename TV>
void size_sweep(SweepPlan& P) {
  constexpr int LW = ColsLanes<TM>::LW, C = LW * Vec16<TM>::N;
  P.smem = (size_t(P.xs_elems) + (256 / LW) * (C + 1)) * sizeof(TV);
  GDSW_CHECK(P.smem <= size_t(200) * 1024, GDSW_ERR_INVALID_ARG, "persistent sweep: staging exceeds shared memory");
  // one limit for every level's launch of this instantiation (the attribute is per kernel)
  GDSW_CUDA(cudaFuncSetAttribute(k_sweep<TM, TV, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  GDSW_CUDA(cudaFuncSetAttribute(k_sweep<TM, TV, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  GDSW_CUDA(cudaFuncSetAttribute(k_sweep<TM, TV, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  int per_sm = 0, dev = 0, nsm = 0;
  if (P.G == 4)
    GDSW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<TM, TV, 4>, 256, P.smem));
  else if (P.G == 2)
    GDSW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<TM, TV, 2>, 256, P.smem));
  else
    GDSW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<TM, TV, 1>, 256, P.smem));
  GDSW_CUDA(cudaGetDevice(&dev));
  GDSW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  GDSW_CHECK(per_sm > 0, GDSW_ERR_CUDA, "persistent sweep: no CTA fits on an SM");
  P.max_per_sm = per_sm;
  const int want = P.ctas_per_sm > 0 ? std::min(P.ctas_per_sm, per_sm) : per_sm;
  P.grid = int(std::min<int64_t>(int64_t(want) * nsm, P.nitems));
}

template <typename TM, typename TV>
void launch_sweep(const TM* M, TV* vec, const SweepPlan& P, unsigned* flag, int T, cudaStream_t s) {
  if (P.nitems == 0) return;
  GDSW_CUDA(cudaMemsetAsync(P.d_ctr, 0, sizeof(unsigned) * P.nctr, s));
  if (P.G == 4)
    k_sweep<TM, TV, 4><<<P.grid, 256, P.smem, s>>>(M, vec, P.d_tasks, P.d_items, P.nitems, P.d_ctr, flag, T,
                                                   P.xs_elems, kSweepWaitLimitNs);
  else if (P.G == 2)
    k_sweep<TM, TV, 2><<<P.grid, 256, P.smem, s>>>(M, vec, P.d_tasks, P.d_items, P.nitems, P.d_ctr, flag, T,
                                                   P.xs_elems, kSweepWaitLimitNs);
  else
    k_sweep<TM, TV, 1><<<P.grid, 256, P.smem, s>>>(M, vec, P.d_tasks, P.d_items, P.nitems, P.d_ctr, flag, T,
                                                   P.xs_elems, kSweepWaitLimitNs);
  check_launch("k_sweep");
}
template void size_sweep<double, double>(SweepPlan&);
template void size_sweep<float, float>(SweepPlan&);
template void size_sweep<__nv_bfloat16, float>(SweepPlan&);
template void launch_sweep<double, double>(const double*, double*, const SweepPlan&, unsigned*, int, cudaStream_t);
template void launch_sweep<float, float>(const float*, float*, const SweepPlan&, unsigned*, int, cudaStream_t);
template void launch_sweep<__nv_bfloat16, float>(const __nv_bfloat16*, float*, const SweepPlan&, unsigned*, int,
                                                 cudaStream_t);

// copy of T x T tiles out of full row-major blocks, zero padded (packing of the upper triangle)
template <typename T>
__global__ void k_pack_tiles(const T* __restrict__ src, T* __restrict__ dst, const PackTile* __restrict__ tiles,
                             int TT) {
  const PackTile p = tiles[blockIdx.x];
  for (int e = threadIdx.x; e < TT * TT; e += blockDim.x) {
    int r = e / TT, c = e - r * TT;
    dst[p.dst + e] = (r < p.rows && c < p.cols) ? src[p.src + int64_t(r) * p.ld + c] : T(0);
  }
}

template <typename T>
void pack_tiles(DevArena& tmp, const T* src, T* dst, const std::vector<PackTile>& tiles, int TT, cudaStream_t s) {
  if (tiles.empty()) return;
  PackTile* d = tmp.upload(tiles, s);
  for (size_t off = 0; off < tiles.size(); off += (size_t(1) << 30)) {
    int nb = int(std::min<size_t>(tiles.size() - off, size_t(1) << 30));
    k_pack_tiles<T><<<nb, 256, 0, s>>>(src, dst, d + off, TT);
    check_launch("k_pack_tiles");
  }
}
template void pack_tiles<double>(DevArena&, const double*, double*, const std::vector<PackTile>&, int, cudaStream_t);
template void pack_tiles<float>(DevArena&, const float*, float*, const std::vector<PackTile>&, int, cudaStream_t);

template void launch_gemv<double, double>(const double*, const double*, double*, const double*, const GemvPlan&,
                                          int, int, cudaStream_t);
template void launch_gemv<float, float>(const float*, const float*, float*, const float*, const GemvPlan&, int,
                                        int, cudaStream_t);
template void launch_gemv<__nv_bfloat16, float>(const __nv_bfloat16*, const float*, float*, const float*,
                                                const GemvPlan&, int, int, cudaStream_t);

void set_gemv_smem_limits() {
  cudaFuncSetAttribute(k_gemv<double, double, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_gemv<float, float, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_gemv<__nv_bfloat16, float, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_gemv<double, double, 4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_gemv<float, float, 4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_gemv<__nv_bfloat16, float, 4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_gemv<double, double, 4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_gemv<float, float, 4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_gemv<__nv_bfloat16, float, 4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_gemvt<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 180 * 1024);
  cudaFuncSetAttribute(k_gemvt<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 180 * 1024);
  cudaFuncSetAttribute(k_gemvt<__nv_bfloat16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 180 * 1024);
}

// ------------------------------------------------------------------ batched GEMM (set-up)
// 64x64 output tile per CTA, 256 threads computing 4x4 each, K staged 16 at a time.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm(const GemmTaskP* __restrict__ tasks, const int32_t* __restrict__ tile_task,
                                              const int32_t* __restrict__ tile_id) {
  __shared__ T As[16][64 + 1];
  __shared__ T Bs[16][64 + 1];
  const GemmTaskP t = tasks[tile_task[blockIdx.x]];
  const int tiles_n = (t.N + 63) / 64;
  const int tm = tile_id[blockIdx.x] / tiles_n, tn = tile_id[blockIdx.x] % tiles_n;
  const T* A = static_cast<const T*>(t.a);
  const T* B = static_cast<const T*>(t.b);
  T* C = static_cast<T*>(t.c);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4] = {};
  for (int k0 = 0; k0 < t.K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      int kk = e / 64, mm = e % 64;
      int gm = tm * 64 + mm, gk = k0 + kk;
      T v = T(0);
      if (gm < t.M && gk < t.K) v = t.ta ? A[int64_t(gk) * t.lda + gm] : A[int64_t(gm) * t.lda + gk];
      As[kk][mm] = v;
      int gn = tn * 64 + mm;
      T w = T(0);
      if (gn < t.N && gk < t.K) w = t.tb ? B[int64_t(gn) * t.ldb + gk] : B[int64_t(gk) * t.ldb + gn];
      Bs[kk][mm] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = tm * 64 + ty * 4 + i;
    if (gm >= t.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = tn * 64 + tx * 4 + j;
      if (gn >= t.N) continue;
      T* cp = C + int64_t(gm) * t.ldc + gn;
      T v = T(t.alpha) * acc[i][j];
      if (t.beta != 0.0) v += T(t.beta) * *cp;
      *cp = v;
    }
  }
}

// ------------------------------------------------------------------ FP32 GEMM tiles
// 128 x 128 outputs per CTA of 256 threads, 8 x 8 per thread (rows ty*4 + {0..3} and
// 64 + ty*4 + {0..3}, columns likewise with tx), K in steps of 16 staged transposed in
// shared memory; the next step's global loads are held in registers while the current
// step is multiplied (one barrier per step).  op(A)(r, k) = ta ? A[k*lda + r] : A[r*lda + k],
// op(B)(k, c) = tb ? B[c*ldb + k] : B[k*ldb + c].
struct GemmOp {
  const float* p;
  int ld, trans;
};

__device__ __forceinline__ void gemm_fetch(const GemmOp& A, const GemmOp& B, int M, int N, int K, int m0, int n0,
                                           int k0, float (&ra)[8], float (&rb)[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int e = threadIdx.x + 256 * i;
    int m, k;
    if (A.trans) { k = e >> 7; m = e & 127; } else { m = e >> 4; k = e & 15; }
    const int gm = m0 + m, gk = k0 + k;
    ra[i] = (gm < M && gk < K) ? (A.trans ? A.p[int64_t(gk) * A.ld + gm] : A.p[int64_t(gm) * A.ld + gk]) : 0.f;
    int c, kk;
    if (B.trans) { c = e >> 4; kk = e & 15; } else { kk = e >> 7; c = e & 127; }
    const int gc = n0 + c, gk2 = k0 + kk;
    rb[i] = (gc < N && gk2 < K) ? (B.trans ? B.p[int64_t(gc) * B.ld + gk2] : B.p[int64_t(gk2) * B.ld + gc]) : 0.f;
  }
}

__device__ __forceinline__ void gemm_stash(const GemmOp& A, const GemmOp& B, const float (&ra)[8],
                                           const float (&rb)[8], float (*As)[132], float (*Bs)[132]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int e = threadIdx.x + 256 * i;
    if (A.trans) As[e >> 7][e & 127] = ra[i]; else As[e & 15][e >> 4] = ra[i];
    if (B.trans) Bs[e & 15][e >> 4] = rb[i]; else Bs[e >> 7][e & 127] = rb[i];
  }
}

// acc = op(A)[m0:, :K] op(B)[:K, n0:] for the CTA's 128 x 128 tile
__device__ __forceinline__ void gemm_tile_f32(const GemmOp& A, const GemmOp& B, int M, int N, int K, int m0, int n0,
                                              float (*As)[16][132], float (*Bs)[16][132], float (&acc)[8][8]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float ra[8], rb[8];
  gemm_fetch(A, B, M, N, K, m0, n0, 0, ra, rb);
  gemm_stash(A, B, ra, rb, As[0], Bs[0]);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const bool more = k0 + 16 < K;
    if (more) gemm_fetch(A, B, M, N, K, m0, n0, k0 + 16, ra, rb);
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) gemm_stash(A, B, ra, rb, As[buf ^ 1], Bs[buf ^ 1]);
    __syncthreads();
    buf ^= 1;
  }
}

__device__ __forceinline__ int gemm_row(int i) { return i < 4 ? (threadIdx.x >> 4) * 4 + i : 64 + (threadIdx.x >> 4) * 4 + i - 4; }
__device__ __forceinline__ int gemm_col(int j) { return j < 4 ? (threadIdx.x & 15) * 4 + j : 64 + (threadIdx.x & 15) * 4 + j - 4; }

__global__ void __launch_bounds__(256, 2) k_gemm_f32(const GemmTaskP* __restrict__ tasks,
                                                  const int32_t* __restrict__ tile_task,
                                                  const int32_t* __restrict__ tile_id) {
  __shared__ __align__(16) float As[2][16][132];
  __shared__ __align__(16) float Bs[2][16][132];
  const GemmTaskP t = tasks[tile_task[blockIdx.x]];
  const int tiles_n = (t.N + 127) / 128;
  const int m0 = (tile_id[blockIdx.x] / tiles_n) * 128, n0 = (tile_id[blockIdx.x] % tiles_n) * 128;
  const GemmOp A{static_cast<const float*>(t.a), t.lda, t.ta};
  const GemmOp B{static_cast<const float*>(t.b), t.ldb, t.tb};
  float acc[8][8];
  gemm_tile_f32(A, B, t.M, t.N, t.K, m0, n0, As, Bs, acc);
  float* C = static_cast<float*>(t.c);
  const float alpha = float(t.alpha), beta = float(t.beta);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + gemm_row(i);
    if (gm >= t.M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gn = n0 + gemm_col(j);
      if (gn >= t.N) continue;
      float* cp = C + int64_t(gm) * t.ldc + gn;
      float v = alpha * acc[i][j];
      if (beta != 0.f) v = fmaf(beta, *cp, v);
      *cp = v;
    }
  }
}

// Which kernel takes the FP32 tasks of 96 x 96 outputs and more: the tensor cores (3xTF32,
// tc_gemm.cu; the default) or the SIMT 128 x 128 tiles below.
static int g_gemm_engine = GDSW_GEMM_AUTO;
void set_gemm_engine(int e) { g_gemm_engine = e; }
int gemm_engine() { return g_gemm_engine; }

template <typename T>
void run_gemm(DevArena& tmp, const std::vector<GemmTaskP>& tasks, cudaStream_t s) {
  run_gemm_engine<T>(tmp, tasks, s, g_gemm_engine);
}

template <typename T>
void run_gemm_engine(DevArena& tmp, const std::vector<GemmTaskP>& tasks, cudaStream_t s, int engine) {
  if (tasks.empty()) return;
  std::vector<int32_t> tt, ti, bt, bi;  // 64-tiles (k_gemm), 128-tiles (k_gemm_f32)
  std::vector<GemmTaskP> tc;             // tasks for the tensor cores
  for (size_t q = 0; q < tasks.size(); ++q) {
    const auto& t = tasks[q];
    if (t.M <= 0 || t.N <= 0) continue;
    if (sizeof(T) == 4 && t.M >= 96 && t.N >= 96 && t.K >= 1 && engine != GDSW_GEMM_SIMT) {
      tc.push_back(t);
      continue;
    }
    if (sizeof(T) == 4 && t.M >= 96 && t.N >= 96) {
      int nt = ((t.M + 127) / 128) * ((t.N + 127) / 128);
      for (int i = 0; i < nt; ++i) {
        bt.push_back(int32_t(q));
        bi.push_back(i);
      }
      continue;
    }
    int nt = ((t.M + 63) / 64) * ((t.N + 63) / 64);
    for (int i = 0; i < nt; ++i) {
      tt.push_back(int32_t(q));
      ti.push_back(i);
    }
  }
  if (!tc.empty()) run_gemm_tc(tc, s);
  if (tt.empty() && bt.empty()) return;
  GemmTaskP* d_t = tmp.upload(tasks, s);
  if (!tt.empty()) {
    int32_t* d_tt = tmp.upload(tt, s);
    int32_t* d_ti = tmp.upload(ti, s);
    k_gemm<T><<<int(tt.size()), 256, 0, s>>>(d_t, d_tt, d_ti);
    check_launch("k_gemm");
  }
  if (!bt.empty()) {
    int32_t* d_bt = tmp.upload(bt, s);
    int32_t* d_bi = tmp.upload(bi, s);
    k_gemm_f32<<<int(bt.size()), 256, 0, s>>>(d_t, d_bt, d_bi);
    check_launch("k_gemm_f32");
  }
}
template void run_gemm<double>(DevArena&, const std::vector<GemmTaskP>&, cudaStream_t);
template void run_gemm<float>(DevArena&, const std::vector<GemmTaskP>&, cudaStream_t);
template void run_gemm_engine<float>(DevArena&, const std::vector<GemmTaskP>&, cudaStream_t, int);

// ------------------------------------------------------------------ batched Gauss-Jordan inverse
// In-place inversion of square blocks with partial pivoting, blocked by panels of NB
// columns: (1) LU with partial pivoting of the remaining rows of the panel chooses the
// pivot rows, (2) those rows are swapped into place, (3) the NB x NB pivot block D is
// inverted, (4) the block sweep A_PP <- D^-1, A_Pj <- D^-1 A_Pj, A_iP <- -A_iP D^-1,
// A_ij <- A_ij - A_iP D^-1 A_Pj is applied as a rank-NB update, and (5) at the end the
// columns are permuted back in reverse pivot order.
constexpr int GJ_NB = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_gj_panel(const InvTaskP* tasks, int kb, T* scratch, int64_t scr_stride,
                                                  int32_t* piv, int64_t piv_stride, double* minpiv) {
  const InvTaskP t = tasks[blockIdx.x];
  if (kb >= t.n) return;
  T* A = static_cast<T*>(t.a);
  const int w = min(GJ_NB, t.n - kb), rows = t.n - kb;
  T* P = scratch + int64_t(t.id) * scr_stride;  // rows x GJ_NB
  int32_t* pv = piv + int64_t(t.id) * piv_stride;
  for (int e = threadIdx.x; e < rows * w; e += blockDim.x) {
    int r = e / w, c = e % w;
    P[int64_t(r) * GJ_NB + c] = A[int64_t(kb + r) * t.ld + kb + c];
  }
  __syncthreads();
  __shared__ double bv[256];
  __shared__ int bi[256];
  __shared__ T prow[GJ_NB];
  for (int j = 0; j < w; ++j) {
    double best = -1.0;
    int besti = rows;
    for (int r = j + threadIdx.x; r < rows; r += blockDim.x) {
      double a = fabs(double(P[int64_t(r) * GJ_NB + j]));
      if (a > best) { best = a; besti = r; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        double a = bv[threadIdx.x + o];
        int ia = bi[threadIdx.x + o];
        if (a > bv[threadIdx.x] || (a == bv[threadIdx.x] && ia < bi[threadIdx.x])) {
          bv[threadIdx.x] = a;
          bi[threadIdx.x] = ia;
        }
      }
      __syncthreads();
    }
    const int p = bi[0];
    const double pmag = bv[0];
    if (threadIdx.x == 0) {
      pv[kb + j] = kb + p;
      if (pmag < minpiv[t.id]) minpiv[t.id] = pmag;
    }
    // swap rows j and p of the panel copy
    if (p != j)
      for (int c = threadIdx.x; c < w; c += blockDim.x) {
        T a = P[int64_t(j) * GJ_NB + c];
        P[int64_t(j) * GJ_NB + c] = P[int64_t(p) * GJ_NB + c];
        P[int64_t(p) * GJ_NB + c] = a;
      }
    __syncthreads();
    for (int c = threadIdx.x; c < w; c += blockDim.x) prow[c] = P[int64_t(j) * GJ_NB + c];
    __syncthreads();
    T d = prow[j];
    if (d == T(0)) d = T(1);  // singular: recorded through minpiv, keep the numbers finite
    for (int r = j + 1 + threadIdx.x; r < rows; r += blockDim.x) {
      T* pr = P + int64_t(r) * GJ_NB;
      T l = pr[j] / d;
      pr[j] = l;
      for (int c = j + 1; c < w; ++c) pr[c] -= l * prow[c];
    }
    __syncthreads();
  }
}

// Pivot choice for one panel, faster form: 1024 threads; the first RS rows of the panel copy
// live in shared memory (row stride NB + 1), the rest in the global scratch; the column
// maximum is found with warp shuffles (largest magnitude, smallest row on ties -- the same
// pivots as the tree reduction above), and the rank-1 elimination runs one warp per row,
// lane = column.  Only the pivot rows are used afterwards.
template <typename T>
__device__ __forceinline__ T& panel_at(T* Ps, T* Pg, int RS, int r, int c) {
  return r < RS ? Ps[r * (GJ_NB + 1) + c] : Pg[int64_t(r) * GJ_NB + c];
}

template <typename T>
__global__ void __launch_bounds__(1024) k_gj_panel_fast(const InvTaskP* tasks, int kb, T* scratch, int64_t scr_stride,
                                                       int32_t* piv, int64_t piv_stride, double* minpiv, int RS) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ps = reinterpret_cast<T*>(smem_raw);
  __shared__ double wv[32];
  __shared__ int wi[32];
  __shared__ int s_p;
  __shared__ T prow[GJ_NB];
  const InvTaskP t = tasks[blockIdx.x];
  if (kb >= t.n) return;
  const T* A = static_cast<const T*>(t.a);
  const int w = min(GJ_NB, t.n - kb), rows = t.n - kb;
  T* Pg = scratch + int64_t(t.id) * scr_stride;
  int32_t* pv = piv + int64_t(t.id) * piv_stride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < rows * w; e += blockDim.x) {
    const int r = e / w, c = e - r * w;
    panel_at(Ps, Pg, RS, r, c) = A[int64_t(kb + r) * t.ld + kb + c];
  }
  __syncthreads();
  for (int j = 0; j < w; ++j) {
    double best = -1.0;
    int bi = rows;
    for (int r = j + threadIdx.x; r < rows; r += blockDim.x) {
      const double a = fabs(double(panel_at(Ps, Pg, RS, r, j)));
      if (a > best) { best = a; bi = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { wv[warp] = best; wi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      const int nw = int(blockDim.x >> 5);
      double b = lane < nw ? wv[lane] : -2.0;
      int i = lane < nw ? wi[lane] : rows;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, b, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ob > b || (ob == b && oi < i)) { b = ob; i = oi; }
      }
      if (lane == 0) {
        s_p = i;
        pv[kb + j] = kb + i;
        if (b < minpiv[t.id]) minpiv[t.id] = b;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p != j && threadIdx.x < w) {
      T& x = panel_at(Ps, Pg, RS, j, threadIdx.x);
      T& y = panel_at(Ps, Pg, RS, p, threadIdx.x);
      const T tmp = x;
      x = y;
      y = tmp;
    }
    __syncthreads();
    if (threadIdx.x < w) prow[threadIdx.x] = panel_at(Ps, Pg, RS, j, threadIdx.x);
    __syncthreads();
    T d = prow[j];
    if (d == T(0)) d = T(1);  // singular: recorded through minpiv, keep the numbers finite
    const int nw = int(blockDim.x >> 5);
    const T pl = lane < w ? prow[lane] : T(0);
    int r = j + 1 + warp;
    for (; r + 3 * nw < rows; r += 4 * nw) {  // four rows of this warp in flight
      T l[4], v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        l[q] = panel_at(Ps, Pg, RS, r + q * nw, j);
        v[q] = lane < w ? panel_at(Ps, Pg, RS, r + q * nw, lane) : T(0);
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T lq = l[q] / d;
        if (lane == j)
          panel_at(Ps, Pg, RS, r + q * nw, j) = lq;
        else if (lane > j && lane < w)
          panel_at(Ps, Pg, RS, r + q * nw, lane) = v[q] - lq * pl;
      }
    }
    for (; r < rows; r += nw) {
      const T l = panel_at(Ps, Pg, RS, r, j) / d;
      __syncwarp();
      if (lane == j)
        panel_at(Ps, Pg, RS, r, j) = l;
      else if (lane > j && lane < w)
        panel_at(Ps, Pg, RS, r, lane) -= l * pl;
    }
    __syncthreads();
  }
}

// swap the chosen pivot rows into place across the full width of the matrix
template <typename T>
__global__ void k_gj_swap(const InvTaskP* tasks, int kb, const int32_t* piv, int64_t piv_stride) {
  const InvTaskP t = tasks[blockIdx.y];
  if (kb >= t.n) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= t.n) return;
  T* A = static_cast<T*>(t.a);
  const int32_t* pv = piv + int64_t(t.id) * piv_stride;
  const int w = min(GJ_NB, t.n - kb);
  for (int j = 0; j < w; ++j) {
    int p = pv[kb + j];
    if (p != kb + j) {
      T a = A[int64_t(kb + j) * t.ld + c];
      A[int64_t(kb + j) * t.ld + c] = A[int64_t(p) * t.ld + c];
      A[int64_t(p) * t.ld + c] = a;
    }
  }
}

// invert the w x w pivot block (pivot order fixed by the panel LU, so no further pivoting)
template <typename T>
__global__ void __launch_bounds__(256) k_gj_dinv(const InvTaskP* tasks, int kb, T* dinv) {
  const InvTaskP t = tasks[blockIdx.x];
  if (kb >= t.n) return;
  const T* A = static_cast<const T*>(t.a);
  const int w = min(GJ_NB, t.n - kb);
  __shared__ T D[GJ_NB][GJ_NB + 1];
  __shared__ T colk[GJ_NB], rk[GJ_NB];
  for (int e = threadIdx.x; e < GJ_NB * GJ_NB; e += blockDim.x) {
    int r = e / GJ_NB, c = e % GJ_NB;
    D[r][c] = (r < w && c < w) ? A[int64_t(kb + r) * t.ld + kb + c] : T(r == c ? 1 : 0);
  }
  __syncthreads();
  const int r0 = threadIdx.x / GJ_NB, c = threadIdx.x % GJ_NB;  // 8 rows x 32 cols per pass
  for (int k = 0; k < w; ++k) {
    if (threadIdx.x < GJ_NB) {
      colk[threadIdx.x] = D[threadIdx.x][k];
      rk[threadIdx.x] = D[k][threadIdx.x];
    }
    __syncthreads();
    T p = rk[k];
    if (p == T(0)) p = T(1);
    const T inv = T(1) / p;
    for (int rr = r0; rr < GJ_NB; rr += 8) {
      T v;
      if (rr == k) v = (c == k) ? inv : rk[c] * inv;
      else v = (c == k) ? -colk[rr] * inv : D[rr][c] - colk[rr] * rk[c] * inv;
      D[rr][c] = v;
    }
    __syncthreads();
  }
  T* out = dinv + int64_t(t.id) * GJ_NB * GJ_NB;
  for (int e = threadIdx.x; e < GJ_NB * GJ_NB; e += blockDim.x) out[e] = D[e / GJ_NB][e % GJ_NB];
}

// Fp = D^-1 A[P, :] (w x n) and E = A[:, P] (n x w) saved before the update
template <typename T>
__global__ void k_gj_fe(const InvTaskP* tasks, int kb, const T* dinv, T* Fp, T* E, int64_t stride) {
  const InvTaskP t = tasks[blockIdx.y];
  if (kb >= t.n) return;
  const T* A = static_cast<const T*>(t.a);
  const int w = min(GJ_NB, t.n - kb);
  const T* Di = dinv + int64_t(t.id) * GJ_NB * GJ_NB;
  T* F = Fp + int64_t(t.id) * stride;
  T* Ee = E + int64_t(t.id) * stride;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= t.n) return;
  // column idx of Fp
  T col[GJ_NB];
#pragma unroll
  for (int q = 0; q < GJ_NB; ++q) col[q] = q < w ? A[int64_t(kb + q) * t.ld + idx] : T(0);
  for (int r = 0; r < w; ++r) {
    T s = T(0);
#pragma unroll
    for (int q = 0; q < GJ_NB; ++q) s = fma(Di[r * GJ_NB + q], col[q], s);
    F[int64_t(r) * t.ld + idx] = s;
  }
  // row idx of E
#pragma unroll
  for (int q = 0; q < GJ_NB; ++q) Ee[int64_t(idx) * GJ_NB + q] = q < w ? A[int64_t(idx) * t.ld + kb + q] : T(0);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gj_update(const InvTaskP* tasks, const int32_t* tile_task,
                                                   const int32_t* tile_id, int kb, const T* dinv, const T* Fp,
                                                   const T* E, int64_t stride) {
  const InvTaskP t = tasks[tile_task[blockIdx.x]];
  if (kb >= t.n) return;
  T* A = static_cast<T*>(t.a);
  const int w = min(GJ_NB, t.n - kb);
  const int tiles = (t.n + 63) / 64;
  const int ti = tile_id[blockIdx.x] / tiles, tj = tile_id[blockIdx.x] % tiles;
  const T* Di = dinv + int64_t(t.id) * GJ_NB * GJ_NB;
  const T* F = Fp + int64_t(t.id) * stride;
  const T* Ee = E + int64_t(t.id) * stride;
  __shared__ T Es[64][GJ_NB + 1];
  __shared__ T Fs[GJ_NB][64 + 1];
  __shared__ T Ds[GJ_NB][GJ_NB + 1];
  for (int e = threadIdx.x; e < 64 * GJ_NB; e += 256) {
    int r = e / GJ_NB, q = e % GJ_NB;
    int gi = ti * 64 + r;
    Es[r][q] = (gi < t.n) ? Ee[int64_t(gi) * GJ_NB + q] : T(0);
    int q2 = e / 64, c = e % 64;
    int gj = tj * 64 + c;
    Fs[q2][c] = (gj < t.n && q2 < w) ? F[int64_t(q2) * t.ld + gj] : T(0);
  }
  for (int e = threadIdx.x; e < GJ_NB * GJ_NB; e += 256) Ds[e / GJ_NB][e % GJ_NB] = Di[e];
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int li = ty * 4 + a, gi = ti * 64 + li;
    if (gi >= t.n) continue;
    bool pi = gi >= kb && gi < kb + w;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int lj = tx * 4 + b, gj = tj * 64 + lj;
      if (gj >= t.n) continue;
      bool pj = gj >= kb && gj < kb + w;
      T* ap = A + int64_t(gi) * t.ld + gj;
      if (pi && pj) {
        *ap = Ds[gi - kb][gj - kb];
      } else if (pi) {
        *ap = Fs[gi - kb][lj];
      } else if (pj) {
        T s = T(0);
        for (int q = 0; q < w; ++q) s = fma(Es[li][q], Ds[q][gj - kb], s);
        *ap = -s;
      } else {
        T s = *ap;
        for (int q = 0; q < w; ++q) s = fma(-Es[li][q], Fs[q][lj], s);
        *ap = s;
      }
    }
  }
}

// FP32 rank-NB sweep on 128 x 128 tiles.  The sweep is bound by the read-modify-write of A,
// so every global load of a tile is issued at once: the A tile and F = D^-1 A[P, :] go to
// shared memory with cp.async, E = A[:, P] (taken before the sweep) is staged transposed; one
// barrier, then the 8 x 8 register-tiled product E F and the epilogue with the four cases of
// the block Gauss-Jordan step (pivot block D^-1, pivot rows F, pivot columns -E D^-1, the rest
// A - E F).  F has the leading dimension of the matrix, so every row starts 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

constexpr int GJU_LD = 132;  // shared row stride (floats) of the update tiles
constexpr size_t GJU_SMEM = size_t(128 + 32 + 32) * GJU_LD * sizeof(float);

__global__ void __launch_bounds__(256, 2) k_gj_update_f32(const InvTaskP* __restrict__ tasks,
                                                          const int32_t* __restrict__ tile_task,
                                                          const int32_t* __restrict__ tile_id, int kb,
                                                          const float* __restrict__ dinv, const float* __restrict__ Fp,
                                                          const float* __restrict__ E, int64_t stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Cs = reinterpret_cast<float*>(smem_raw);  // 128 x GJU_LD
  float* Es = Cs + 128 * GJU_LD;                   // 32 x GJU_LD, Es[k][m] = E[m0 + m][k]
  float* Fs = Es + 32 * GJU_LD;                    // 32 x GJU_LD, Fs[k][c] = F[k][n0 + c]
  __shared__ float Ds[GJ_NB][GJ_NB + 1];
  const InvTaskP t = tasks[tile_task[blockIdx.x]];
  if (kb >= t.n) return;
  const int w = min(GJ_NB, t.n - kb);
  const int tiles = (t.n + 127) / 128;
  const int m0 = (tile_id[blockIdx.x] / tiles) * 128, n0 = (tile_id[blockIdx.x] % tiles) * 128;
  const float* Di = dinv + int64_t(t.id) * GJ_NB * GJ_NB;
  const float* F = Fp + int64_t(t.id) * stride;
  const float* Ee = E + int64_t(t.id) * stride;
  float* Am = static_cast<float*>(t.a);
  const int nch = min(32, (t.ld - n0) / 4);  // 16-byte chunks of a tile row inside the padded row
  for (int e = threadIdx.x; e < 128 * 32; e += 256) {  // A tile
    const int r = e >> 5, ch = e & 31;
    if (m0 + r < t.n && ch < nch) cp_async16(Cs + r * GJU_LD + ch * 4, Am + int64_t(m0 + r) * t.ld + n0 + ch * 4);
  }
  for (int e = threadIdx.x; e < 32 * 32; e += 256) {  // F tile
    const int k = e >> 5, ch = e & 31;
    if (k < w && ch < nch) cp_async16(Fs + k * GJU_LD + ch * 4, F + int64_t(k) * t.ld + n0 + ch * 4);
  }
  for (int e = threadIdx.x; e < 128 * 8; e += 256) {  // E tile, transposed
    const int r = e >> 3, q = (e & 7) * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m0 + r < t.n) v = *reinterpret_cast<const float4*>(Ee + int64_t(m0 + r) * GJ_NB + q);
    Es[(q + 0) * GJU_LD + r] = v.x;
    Es[(q + 1) * GJU_LD + r] = v.y;
    Es[(q + 2) * GJU_LD + r] = v.z;
    Es[(q + 3) * GJU_LD + r] = v.w;
  }
  for (int e = threadIdx.x; e < GJ_NB * GJ_NB; e += 256) Ds[e / GJ_NB][e % GJ_NB] = Di[e];
  cp_async_wait_all();
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  for (int k = 0; k < w; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(Es + k * GJU_LD + ty * 4);
    const float4 a1 = *reinterpret_cast<const float4*>(Es + k * GJU_LD + 64 + ty * 4);
    const float4 b0 = *reinterpret_cast<const float4*>(Fs + k * GJU_LD + tx * 4);
    const float4 b1 = *reinterpret_cast<const float4*>(Fs + k * GJU_LD + 64 + tx * 4);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int li = gemm_row(i), gi = m0 + li;
    if (gi >= t.n) continue;
    const bool pi = gi >= kb && gi < kb + w;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int lj = gemm_col(j), gj = n0 + lj;
      if (gj >= t.n) continue;
      const bool pj = gj >= kb && gj < kb + w;
      float v;
      if (pi && pj) {
        v = Ds[gi - kb][gj - kb];
      } else if (pi) {
        v = Fs[(gi - kb) * GJU_LD + lj];
      } else if (pj) {
        float sum = 0.f;
        for (int q = 0; q < w; ++q) sum = fmaf(Es[q * GJU_LD + li], Ds[q][gj - kb], sum);
        v = -sum;
      } else {
        v = Cs[li * GJU_LD + lj] - acc[i][j];
      }
      Am[int64_t(gi) * t.ld + gj] = v;
    }
  }
}

template <typename T>
__global__ void k_gj_colperm(const InvTaskP* tasks, const int32_t* piv, int64_t piv_stride) {
  const InvTaskP t = tasks[blockIdx.y];
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= t.n) return;
  T* A = static_cast<T*>(t.a) + int64_t(r) * t.ld;
  const int32_t* pv = piv + int64_t(t.id) * piv_stride;
  for (int j = t.n - 1; j >= 0; --j) {
    int p = pv[j];
    if (p != j) {
      T a = A[j];
      A[j] = A[p];
      A[p] = a;
    }
  }
}

__global__ void k_fill_d(double* p, double v, int64_t n) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) p[i] = v;
}

// Invert every task's matrix in place; returns the smallest pivot magnitude per task.
template <typename T>
void run_inverse(DevArena& tmp, const std::vector<InvTaskP>& tasks_in, std::vector<double>& minpiv,
                 cudaStream_t s) {
  minpiv.assign(tasks_in.size(), 0.0);
  std::vector<InvTaskP> tasks;
  int nmax = 0;
  for (size_t q = 0; q < tasks_in.size(); ++q) {
    InvTaskP t = tasks_in[q];
    t.id = int32_t(q);
    if (t.n > 0) {
      tasks.push_back(t);
      nmax = std::max(nmax, t.n);
    }
  }
  if (tasks.empty()) return;
  const int nt = int(tasks.size());
  const int64_t nq = int64_t(tasks_in.size());
  int ldmax = 8;
  for (const InvTaskP& t : tasks) ldmax = std::max(ldmax, t.ld);
  // F rows have the matrices' leading dimension
  const int64_t stride = std::max<int64_t>(pad8(nmax), ldmax) * GJ_NB;
  T* scratch = tmp.alloc<T>(size_t(nq) * stride);
  T* Fp = tmp.alloc<T>(size_t(nq) * stride);
  T* E = tmp.alloc<T>(size_t(nq) * stride);
  T* dinv = tmp.alloc<T>(size_t(nq) * GJ_NB * GJ_NB);
  int32_t* piv = tmp.alloc<int32_t>(size_t(nq) * nmax);
  double* d_min = tmp.alloc<double>(nq);
  k_fill_d<<<int((nq + 255) / 256), 256, 0, s>>>(d_min, DBL_MAX, nq);
  InvTaskP* d_tasks = tmp.upload(tasks, s);
  const int TE = sizeof(T) == 4 ? 128 : 64;  // update tile edge
  std::vector<int32_t> tt, ti;
  for (int q = 0; q < nt; ++q) {
    int tl = (tasks[q].n + TE - 1) / TE;
    for (int i = 0; i < tl * tl; ++i) {
      tt.push_back(q);
      ti.push_back(i);
    }
  }
  int32_t* d_tt = tmp.upload(tt, s);
  int32_t* d_ti = tmp.upload(ti, s);
  dim3 gcol((nmax + 255) / 256, nt);
  const size_t panel_smem = size_t(200) * 1024;
  const int panel_rs = int(panel_smem / ((GJ_NB + 1) * sizeof(T)));
  GDSW_CUDA(cudaFuncSetAttribute(k_gj_panel_fast<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(panel_smem)));
  GDSW_CUDA(cudaFuncSetAttribute(k_gj_update_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(GJU_SMEM)));
  for (int kb = 0; kb < nmax; kb += GJ_NB) {
    k_gj_panel_fast<T><<<nt, 1024, panel_smem, s>>>(d_tasks, kb, scratch, stride, piv, nmax, d_min, panel_rs);
    k_gj_swap<T><<<gcol, 256, 0, s>>>(d_tasks, kb, piv, nmax);
    k_gj_dinv<T><<<nt, 256, 0, s>>>(d_tasks, kb, dinv);
    k_gj_fe<T><<<gcol, 256, 0, s>>>(d_tasks, kb, dinv, Fp, E, stride);
    if (sizeof(T) == 4)
      k_gj_update_f32<<<int(tt.size()), 256, GJU_SMEM, s>>>(d_tasks, d_tt, d_ti, kb, reinterpret_cast<const float*>(dinv),
                                                     reinterpret_cast<const float*>(Fp),
                                                     reinterpret_cast<const float*>(E), stride);
    else
      k_gj_update<T><<<int(tt.size()), 256, 0, s>>>(d_tasks, d_tt, d_ti, kb, dinv, Fp, E, stride);
    check_launch("gauss-jordan panel");
  }
  k_gj_colperm<T><<<gcol, 256, 0, s>>>(d_tasks, piv, nmax);
  check_launch("k_gj_colperm");
  GDSW_CUDA(cudaMemcpyAsync(minpiv.data(), d_min, sizeof(double) * nq, cudaMemcpyDeviceToHost, s));
  GDSW_CUDA(cudaStreamSynchronize(s));
  for (size_t q = 0; q < tasks_in.size(); ++q)
    if (tasks_in[q].n == 0) minpiv[q] = 1.0;
  tmp.release(scratch); tmp.release(Fp); tmp.release(E); tmp.release(dinv); tmp.release(piv);
  tmp.release(d_min); tmp.release(d_tasks); tmp.release(d_tt); tmp.release(d_ti);
}
template void run_inverse<double>(DevArena&, const std::vector<InvTaskP>&, std::vector<double>&, cudaStream_t);
template void run_inverse<float>(DevArena&, const std::vector<InvTaskP>&, std::vector<double>&, cudaStream_t);

// ------------------------------------------------------------------ conversions
__global__ void k_f64_to_f32(const double* a, float* b, int64_t n) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) b[i] = float(a[i]);
}
__global__ void k_f32_to_f64(const float* a, double* b, int64_t n) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) b[i] = double(a[i]);
}
__global__ void k_f32_to_bf16(const float* a, __nv_bfloat16* b, int64_t n) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}
__global__ void k_f64_to_bf16(const double* a, __nv_bfloat16* b, int64_t n) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(float(a[i]));
}
void convert(const void* src, int sprec, void* dst, int dprec, int64_t n, cudaStream_t s) {
  if (n == 0) return;
  int blocks = int((n + 255) / 256);
  if (sprec == GDSW_FP64 && dprec == GDSW_FP32)
    k_f64_to_f32<<<blocks, 256, 0, s>>>(static_cast<const double*>(src), static_cast<float*>(dst), n);
  else if (sprec == GDSW_FP32 && dprec == GDSW_FP64)
    k_f32_to_f64<<<blocks, 256, 0, s>>>(static_cast<const float*>(src), static_cast<double*>(dst), n);
  else if (sprec == GDSW_FP32 && dprec == GDSW_BF16)
    k_f32_to_bf16<<<blocks, 256, 0, s>>>(static_cast<const float*>(src), static_cast<__nv_bfloat16*>(dst), n);
  else if (sprec == GDSW_FP64 && dprec == GDSW_BF16)
    k_f64_to_bf16<<<blocks, 256, 0, s>>>(static_cast<const double*>(src), static_cast<__nv_bfloat16*>(dst), n);
  else if (sprec == dprec)
    GDSW_CUDA(cudaMemcpyAsync(dst, src, n * elem_size(sprec), cudaMemcpyDeviceToDevice, s));
  else
    throw Error{GDSW_ERR_INVALID_ARG, "unsupported precision conversion"};
  check_launch("convert");
}

}  // namespace gdsw
