// Restarted flexible GMRES (right preconditioning) in FP64 on the device
// (arXiv 2606.01433, Section 3: the linearised system is solved by restarted FGMRES
// preconditioned by the multilevel monolithic Schwarz operator).
// Arnoldi with classical Gram-Schmidt applied twice (CGS2): each pass is one fused
// multi-dot over the basis and one multi-axpy.  All reductions are two-stage with a fixed
// order, so the iteration is bitwise reproducible.  The Hessenberg least-squares problem
// (Givens rotations, back substitution) stays on the device in FP64.
#include <cmath>

#include "common.h"
#include "kernels.h"

namespace gdsw {

void apply_precond(gdsw_ctx* c, const double* r, double* z, cudaStream_t s);

constexpr int RB = 304;     // reduction blocks (2 per SM)
constexpr int RT = 256;
constexpr int DG = 8;       // basis vectors per multi-dot pass

// part[b * ldp + t0 + q] = sum over block b's chunk of V[t0+q][e] * w[e]
__global__ void __launch_bounds__(RT) k_dots(const double* __restrict__ V, int64_t n, int nvec,
                                             const double* __restrict__ w, double* __restrict__ part, int ldp) {
  dep_release();
  dep_wait();
  __shared__ double red[DG][RT];
  const int t0 = blockIdx.y * DG;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = blockIdx.x * chunk, e1 = min(n, e0 + chunk);
  double acc[DG];
#pragma unroll
  for (int q = 0; q < DG; ++q) acc[q] = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += RT) {
    double we = w[e];
#pragma unroll
    for (int q = 0; q < DG; ++q)
      if (t0 + q < nvec) acc[q] = fma(__ldcs(V + int64_t(t0 + q) * n + e), we, acc[q]);
  }
#pragma unroll
  for (int q = 0; q < DG; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int o = RT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int q = 0; q < DG; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < DG && t0 + threadIdx.x < nvec) part[int64_t(blockIdx.x) * ldp + t0 + threadIdx.x] = red[threadIdx.x][0];
}

// out[t] (+)= sum_b part[b * ldp + t]: one warp per t, lane-strided partial sums and a
// fixed butterfly (deterministic)
__global__ void k_sum_parts(const double* __restrict__ part, int nb, int nvec, int ldp, double* __restrict__ out,
                            int accumulate) {
  dep_release();
  dep_wait();
  const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (t >= nvec) return;
  double s = 0.0;
  for (int b = lane; b < nb; b += 32) s += part[int64_t(b) * ldp + t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[t] = accumulate ? out[t] + s : s;
}

// w -= sum_t h[t] V[t]
__global__ void k_update(const double* __restrict__ V, int64_t n, int nvec, const double* __restrict__ h,
                         double* __restrict__ w) {
  dep_release();
  dep_wait();
  extern __shared__ double hs[];
  for (int t = threadIdx.x; t < nvec; t += blockDim.x) hs[t] = h[t];
  __syncthreads();
  int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= n) return;
  double a = w[e];
  for (int t = 0; t < nvec; ++t) a = fma(-hs[t], __ldcs(V + int64_t(t) * n + e), a);
  w[e] = a;
}

// x += sum_t y[t] Z[t]
__global__ void k_xupdate(const double* __restrict__ Z, int64_t n, int nvec, const double* __restrict__ y,
                          double* __restrict__ x) {
  dep_release();
  dep_wait();
  extern __shared__ double ys[];
  for (int t = threadIdx.x; t < nvec; t += blockDim.x) ys[t] = y[t];
  __syncthreads();
  int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= n) return;
  double a = x[e];
  for (int t = 0; t < nvec; ++t) a = fma(ys[t], Z[int64_t(t) * n + e], a);
  x[e] = a;
}

__global__ void k_norm_parts(const double* __restrict__ w, int64_t n, double* __restrict__ part) {
  dep_release();
  dep_wait();
  __shared__ double red[RT];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = blockIdx.x * chunk, e1 = min(n, e0 + chunk);
  double acc = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += RT) acc = fma(w[e], w[e], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = RT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// scal[slot] = sqrt(sum of parts)
__global__ void k_norm_finish(const double* __restrict__ part, int nb, double* __restrict__ scal, int slot) {
  dep_release();
  dep_wait();
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += part[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) scal[slot] = sqrt(s);
}

// v = w / scal[slot] (0 if the norm vanished)
__global__ void k_scale(const double* __restrict__ w, int64_t n, const double* __restrict__ scal, int slot,
                        double* __restrict__ v) {
  dep_release();
  dep_wait();
  int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= n) return;
  double d = scal[slot];
  v[e] = d > 0.0 ? w[e] / d : 0.0;
}

// column j of H (column-major, leading dimension m+1) receives H[j+1][j] = scal[1], then
// the previous rotations, a new rotation, and the updated right-hand side g.  scal[2] =
// |g[j+1]| (the residual estimate), mirrored to pinned host memory.
__global__ void k_givens(double* __restrict__ H, int ldh, int j, double* __restrict__ cs, double* __restrict__ sn,
                         double* __restrict__ g, double* __restrict__ scal, double* __restrict__ hmirror) {
  dep_release();
  dep_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = H + int64_t(j) * ldh;
  col[j + 1] = scal[1];
  for (int i = 0; i < j; ++i) {
    double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  double a = col[j], b = col[j + 1];
  double den = hypot(a, b);
  double c = den > 0.0 ? a / den : 1.0, s = den > 0.0 ? b / den : 0.0;
  cs[j] = c;
  sn[j] = s;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  scal[2] = fabs(g[j + 1]);
  if (hmirror) hmirror[0] = scal[2];
}

// back substitution y = R^{-1} g for the first k columns
__global__ void k_backsolve(const double* __restrict__ H, int ldh, int k, const double* __restrict__ g,
                            double* __restrict__ y) {
  dep_release();
  dep_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < k; ++q) s -= H[int64_t(q) * ldh + i] * y[q];
    double d = H[int64_t(i) * ldh + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

// start of a cycle: V[0] = r / beta, g = (beta, 0, ...)
__global__ void k_cycle_start(double* __restrict__ g, int m1, const double* __restrict__ scal) {
  dep_release();
  dep_wait();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m1) g[t] = t == 0 ? scal[0] : 0.0;
}

static void ensure_workspace(gdsw_ctx* c, int m) {
  if (c->m_alloc >= m) return;
  const int64_t n = c->mesh.n;
  c->d_V = c->arena.alloc<double>((m + 1) * n);
  c->d_Z = c->arena.alloc<double>(m * n);
  c->d_H = c->arena.alloc<double>((m + 1) * int64_t(m + 1));
  c->d_gvec = c->arena.alloc<double>(m + 1);
  c->d_cs = c->arena.alloc<double>(m + 1);
  c->d_sn = c->arena.alloc<double>(m + 1);
  c->d_y = c->arena.alloc<double>(m + 1);
  c->d_part = c->arena.alloc<double>(int64_t(RB) * (m + 2));
  c->d_scal = c->arena.alloc<double>(8);
  c->m_alloc = m;
}

// w <- w - V h twice (CGS2); H column j receives the summed coefficients
static void cgs2(gdsw_ctx* c, int j, double* w, cudaStream_t s) {
  const int64_t n = c->mesh.n;
  const int nvec = j + 1;
  const int ldp = c->m_alloc + 2;
  double* hcol = c->d_H + int64_t(j) * (c->m_alloc + 1);
  dim3 gd(RB, (nvec + DG - 1) / DG);
  const int ub = int((n + 255) / 256);
  // four passes over the basis (two multi-dots, two multi-axpys) plus w traffic and the norm
  ProfScope ps(c, GDSW_K_ARNOLDI, 8.0 * n * (4.0 * nvec + 7.0), s);
  for (int pass = 0; pass < 2; ++pass) {
    launch_chained(k_dots, gd, dim3(RT), 0, s, c->d_V, n, nvec, w, c->d_part, ldp);
    check_launch("k_dots");
    launch_chained(k_sum_parts, dim3((nvec + 3) / 4), dim3(128), 0, s, c->d_part, RB, nvec, ldp,
                   pass == 0 ? hcol : c->d_y, 0);
    check_launch("k_sum_parts");
    launch_chained(k_update, dim3(ub), dim3(256), nvec * sizeof(double), s, c->d_V, n, nvec,
                   pass == 0 ? hcol : c->d_y, w);
    check_launch("k_update");
    if (pass == 1) {
      launch_chained(k_sum_parts, dim3((nvec + 3) / 4), dim3(128), 0, s, c->d_part, RB, nvec, ldp, hcol, 1);
      check_launch("k_sum_parts");
    }
  }
  launch_chained(k_norm_parts, dim3(RB), dim3(RT), 0, s, w, n, c->d_part);
  check_launch("k_norm_parts");
  launch_chained(k_norm_finish, dim3(1), dim3(32), 0, s, c->d_part, RB, c->d_scal, 1);
  check_launch("k_norm_finish");
}

void fgmres_solve(gdsw_ctx* c, const double* b, double* x, gdsw_solve_info* info) {
  cudaStream_t s = c->stream;
  const int64_t n = c->mesh.n;
  const int m = std::max(1, c->opt.restart);
  ensure_workspace(c, m);
  const int ldh = c->m_alloc + 1;
  const int ub = int((n + 255) / 256);
  cudaEvent_t e0, e1;
  GDSW_CUDA(cudaEventCreate(&e0));
  GDSW_CUDA(cudaEventCreate(&e1));
  GDSW_CUDA(cudaEventRecord(e0, s));
  // ||b||
  k_norm_parts<<<RB, RT, 0, s>>>(b, n, c->d_part);
  check_launch("k_norm_parts");
  k_norm_finish<<<1, 32, 0, s>>>(c->d_part, RB, c->d_scal, 3);
  check_launch("k_norm_finish");
  double bnorm = 0.0;
  GDSW_CUDA(cudaMemcpyAsync(&bnorm, c->d_scal + 3, 8, cudaMemcpyDeviceToHost, s));
  GDSW_CUDA(cudaStreamSynchronize(s));
  *info = gdsw_solve_info{};
  if (!(bnorm > 0.0)) {
    GDSW_CUDA(cudaMemsetAsync(x, 0, 8 * n, s));
    info->status = std::isfinite(bnorm) ? GDSW_OK : GDSW_ERR_NAN;
    GDSW_CUDA(cudaStreamSynchronize(s));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return;
  }
  const double tol = c->opt.tol;
  int it = 0;
  double est = 0.0, beta = 0.0;
  const double spmv_b = c->spmv_bytes();
  auto true_residual = [&]() {
    {
      ProfScope ps(c, GDSW_K_SPMV, spmv_b + 8.0 * n, s);
      launch_spmv(c, x, c->d_V, b, s);  // V[0] = b - A x
    }
    k_norm_parts<<<RB, RT, 0, s>>>(c->d_V, n, c->d_part);
    check_launch("k_norm_parts");
    k_norm_finish<<<1, 32, 0, s>>>(c->d_part, RB, c->d_scal, 0);
    check_launch("k_norm_finish");
    GDSW_CUDA(cudaMemcpyAsync(&beta, c->d_scal, 8, cudaMemcpyDeviceToHost, s));
    GDSW_CUDA(cudaStreamSynchronize(s));
  };
  true_residual();
  int status = GDSW_OK;
  while (true) {
    if (!std::isfinite(beta)) {
      status = GDSW_ERR_NAN;
      break;
    }
    if (beta / bnorm <= tol) break;
    if (it >= c->opt.max_it) {
      status = GDSW_ERR_NOT_CONVERGED;
      break;
    }
    k_scale<<<ub, 256, 0, s>>>(c->d_V, n, c->d_scal, 0, c->d_V);
    check_launch("k_scale");
    k_cycle_start<<<(m + 1 + 127) / 128, 128, 0, s>>>(c->d_gvec, m + 1, c->d_scal);
    check_launch("k_cycle_start");
    int jd = 0;
    for (int j = 0; j < m && it < c->opt.max_it; ++j) {
      double* vj = c->d_V + int64_t(j) * n;
      double* zj = c->d_Z + int64_t(j) * n;
      double* w = c->d_V + int64_t(j + 1) * n;
      apply_precond(c, vj, zj, s);
      {
        ProfScope ps(c, GDSW_K_SPMV, spmv_b, s);
        launch_spmv(c, zj, w, nullptr, s);
      }
      cgs2(c, j, w, s);
      launch_chained(k_scale, dim3(ub), dim3(256), 0, s, w, n, c->d_scal, 1, w);
      check_launch("k_scale");
      launch_chained(k_givens, dim3(1), dim3(32), 0, s, c->d_H, ldh, j, c->d_cs, c->d_sn, c->d_gvec, c->d_scal,
                     static_cast<double*>(nullptr));
      check_launch("k_givens");
      GDSW_CUDA(cudaMemcpyAsync(c->h_scal, c->d_scal + 2, 8, cudaMemcpyDeviceToHost, s));
      GDSW_CUDA(cudaStreamSynchronize(s));
      est = c->h_scal[0];
      ++it;
      jd = j + 1;
      if (!std::isfinite(est)) {
        status = GDSW_ERR_NAN;
        break;
      }
      if (est / bnorm <= tol) break;
    }
    if (status == GDSW_ERR_NAN) break;
    k_backsolve<<<1, 32, 0, s>>>(c->d_H, ldh, jd, c->d_gvec, c->d_y);
    check_launch("k_backsolve");
    k_xupdate<<<ub, 256, jd * sizeof(double), s>>>(c->d_Z, n, jd, c->d_y, x);
    check_launch("k_xupdate");
    true_residual();
  }
  GDSW_CUDA(cudaEventRecord(e1, s));
  GDSW_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (c->d_sweep_flag) {  // a persistent sweep gave up waiting: the preconditioner output is void
    unsigned flag = 0;
    GDSW_CUDA(cudaMemcpyAsync(&flag, c->d_sweep_flag, sizeof(flag), cudaMemcpyDeviceToHost, s));
    GDSW_CUDA(cudaStreamSynchronize(s));
    if (flag) {
      GDSW_CUDA(cudaMemsetAsync(c->d_sweep_flag, 0, sizeof(unsigned), s));
      status = GDSW_ERR_TIMEOUT;
      c->err = "persistent local sweep: a dependency wait exceeded its time limit";
    }
  }
  info->iterations = it;
  info->relres = beta / bnorm;
  info->est_relres = est / bnorm;
  info->status = status;
  info->time_ms = ms;
}

}  // namespace gdsw
