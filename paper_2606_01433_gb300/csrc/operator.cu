// The saddle-point operator on the device: Carreau viscosity at the Gauss points, the
// assembly of A_cal = [[A, B^T], [B, 0]], the Dirichlet lifting and the FP64 SpMV.
//   arXiv 2606.01433, Section 2 (weak form, saddle-point equation), Section 3 (Carreau
//   law nu = nu0 (1 + (lambda gamma_dot)^2)^((n-1)/2), gamma_dot = sqrt(2 D:D), here with
//   an infinite-shear offset nu_inf; symmetric form 2 nu D(u):D(v)).
// Storage: 3x3 velocity blocks per (free velocity node, free velocity node) pair sharing
// a fluid element (row-major block, 72 bytes); pressure-velocity entries as 3-vectors in
// both row orientations (B rows per pressure node, B^T rows per velocity node).
#include "common.h"
#include "kernels.h"

namespace gdsw {

void host_tables(RefTables& T) {
  const double gx[3] = {-0.7745966692414834, 0.0, 0.7745966692414834};  // -sqrt(3/5), 0, sqrt(3/5)
  const double gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  auto q2 = [](int a, double x) { return a == 0 ? 0.5 * x * (x - 1.0) : (a == 1 ? 1.0 - x * x : 0.5 * x * (x + 1.0)); };
  auto dq2 = [](int a, double x) { return a == 0 ? x - 0.5 : (a == 1 ? -2.0 * x : x + 0.5); };
  auto q1 = [](int a, double x) { return a == 0 ? 0.5 * (1.0 - x) : 0.5 * (1.0 + x); };
  for (int qz = 0; qz < 3; ++qz)
    for (int qy = 0; qy < 3; ++qy)
      for (int qx = 0; qx < 3; ++qx) {
        int q = qx + 3 * qy + 9 * qz;
        double x = gx[qx], y = gx[qy], z = gx[qz];
        T.w[q] = gw[qx] * gw[qy] * gw[qz];
        T.p1[q][0] = 1.0;
        T.p1[q][1] = x;
        T.p1[q][2] = y;
        T.p1[q][3] = z;
        for (int az = 0; az < 3; ++az)
          for (int ay = 0; ay < 3; ++ay)
            for (int ax = 0; ax < 3; ++ax) {
              int a = ax + 3 * ay + 9 * az;
              T.dphi[q][a][0] = dq2(ax, x) * q2(ay, y) * q2(az, z);
              T.dphi[q][a][1] = q2(ax, x) * dq2(ay, y) * q2(az, z);
              T.dphi[q][a][2] = q2(ax, x) * q2(ay, y) * dq2(az, z);
            }
        for (int pz = 0; pz < 2; ++pz)
          for (int py = 0; py < 2; ++py)
            for (int px = 0; px < 2; ++px) T.psi[q][px + 2 * py + 4 * pz] = q1(px, x) * q1(py, y) * q1(pz, z);
      }
}

struct Geo {
  int nx, ny, nz, NX, NY;
  double h;
};

__device__ __forceinline__ void node_ijk(int64_t v, const Geo& G, int& i, int& j, int& k) {
  i = int(v % G.NX);
  j = int((v / G.NX) % G.NY);
  k = int(v / (int64_t(G.NX) * G.NY));
}

// elements (per axis) containing both node coordinates a and b
__device__ __forceinline__ int shared_range(int a, int b, int n, int& e0) {
  int lo = max(a, b), hi = min(a, b);
  if (lo - hi > 2) return 0;
  e0 = lo < 2 ? 0 : (lo - 1) / 2;
  int e1 = min(n - 1, hi / 2);
  return e1 >= e0 ? e1 - e0 + 1 : 0;
}

// ------------------------------------------------------------------ a1: Carreau viscosity
// dn (optional, Newton linearisation of Section 3): per Gauss point D(u_k) (xx, yy, zz, xy, xz,
// yz) and N = 4 nu'(gamma_dot) / gamma_dot = 4 (nu0 - nu_inf)(n - 1) lambda^2
// (1 + (lambda gamma_dot)^2)^((n - 3)/2), the weight of the Newton term
// int N (D(u_k):D(w)) (D(u_k):D(v)) of the Carreau operator's derivative
__global__ void k_viscosity(const int32_t* __restrict__ fluid, int64_t nfe, const double* __restrict__ uk,
                            const RefTables* __restrict__ T, Geo G, int form, int has_uk, double nu0, double nu_inf,
                            double lam, double ncar, double* __restrict__ nu, double* __restrict__ dn) {
  int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= nfe * 27) return;
  int64_t fe = t / 27;
  int q = int(t - fe * 27);
  if (!has_uk || form == GDSW_FORM_GRADIENT) {
    nu[t] = nu0;
    if (dn)
      for (int k = 0; k < 7; ++k) dn[t * 7 + k] = 0.0;
    return;
  }
  int e = fluid[fe];
  int ex = e % G.nx, ey = (e / G.nx) % G.ny, ez = e / (G.nx * G.ny);
  double gr[3][3] = {};
  for (int a = 0; a < 27; ++a) {
    int ax = a % 3, ay = (a / 3) % 3, az = a / 9;
    int64_t v = (2 * ex + ax) + int64_t(G.NX) * ((2 * ey + ay) + int64_t(G.NY) * (2 * ez + az));
    const double* dp = T->dphi[q][a];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double u = uk[3 * v + c];
#pragma unroll
      for (int l = 0; l < 3; ++l) gr[c][l] = fma(u, dp[l], gr[c][l]);
    }
  }
  const double s = 2.0 / G.h;
  double dd = 0.0;  // D : D
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      double d = 0.5 * s * (gr[c][l] + gr[l][c]);
      dd = fma(d, d, dd);
    }
  double gdot = sqrt(2.0 * dd);
  double lg = lam * gdot;
  nu[t] = nu_inf + (nu0 - nu_inf) * pow(1.0 + lg * lg, 0.5 * (ncar - 1.0));
  if (dn) {
    double* o = dn + t * 7;
    o[0] = s * gr[0][0];
    o[1] = s * gr[1][1];
    o[2] = s * gr[2][2];
    o[3] = 0.5 * s * (gr[0][1] + gr[1][0]);
    o[4] = 0.5 * s * (gr[0][2] + gr[2][0]);
    o[5] = 0.5 * s * (gr[1][2] + gr[2][1]);
    o[6] = 4.0 * (nu0 - nu_inf) * (ncar - 1.0) * lam * lam * pow(1.0 + lg * lg, 0.5 * (ncar - 3.0));
  }
}

// 3x3 velocity block between nodes I and J (Section 2 gradient form / Section 3 symmetric form)
__device__ void velocity_block(int64_t I, int64_t J, const Geo& G, const uint8_t* mask, const int32_t* felem,
                               const double* nu, const RefTables* T, int form, double out[9]) {
  int ii, ij, ik, ji, jj, jk;
  node_ijk(I, G, ii, ij, ik);
  node_ijk(J, G, ji, jj, jk);
#pragma unroll
  for (int c = 0; c < 9; ++c) out[c] = 0.0;
  int e0x, e0y, e0z;
  int nxr = shared_range(ii, ji, G.nx, e0x), nyr = shared_range(ij, jj, G.ny, e0y), nzr = shared_range(ik, jk, G.nz, e0z);
  const double sc = 0.5 * G.h;  // (h/2)^3 * (2/h)^2
  for (int cz = 0; cz < nzr; ++cz)
    for (int cy = 0; cy < nyr; ++cy)
      for (int cx = 0; cx < nxr; ++cx) {
        int ex = e0x + cx, ey = e0y + cy, ez = e0z + cz;
        int64_t e = ex + int64_t(G.nx) * (ey + int64_t(G.ny) * ez);
        if (!mask[e]) continue;
        int fe = felem[e];
        int a = (ii - 2 * ex) + 3 * (ij - 2 * ey) + 9 * (ik - 2 * ez);
        int b = (ji - 2 * ex) + 3 * (jj - 2 * ey) + 9 * (jk - 2 * ez);
        const double* nq = nu + int64_t(fe) * 27;
        for (int q = 0; q < 27; ++q) {
          const double* da = T->dphi[q][a];
          const double* db = T->dphi[q][b];
          double f = nq[q] * T->w[q] * sc;
          double g = da[0] * db[0] + da[1] * db[1] + da[2] * db[2];
          out[0] = fma(f, g, out[0]);
          out[4] = fma(f, g, out[4]);
          out[8] = fma(f, g, out[8]);
          if (form == GDSW_FORM_SYMMETRIC) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
              for (int d = 0; d < 3; ++d) out[c * 3 + d] = fma(f, da[d] * db[c], out[c * 3 + d]);
          }
        }
      }
}

// pressure-velocity entry: -int psi_P d_d phi_J over shared fluid elements, d = 0..2
__device__ void divergence_entry(int64_t P, int64_t J, const Geo& G, const uint8_t* mask, const RefTables* T,
                                 double out[3]) {
  int pi, pj, pk, ji, jj, jk;
  node_ijk(P, G, pi, pj, pk);
  node_ijk(J, G, ji, jj, jk);
  out[0] = out[1] = out[2] = 0.0;
  int e0x, e0y, e0z;
  int nxr = shared_range(pi, ji, G.nx, e0x), nyr = shared_range(pj, jj, G.ny, e0y), nzr = shared_range(pk, jk, G.nz, e0z);
  const double sc = 0.25 * G.h * G.h;  // (h/2)^3 * (2/h)
  for (int cz = 0; cz < nzr; ++cz)
    for (int cy = 0; cy < nyr; ++cy)
      for (int cx = 0; cx < nxr; ++cx) {
        int ex = e0x + cx, ey = e0y + cy, ez = e0z + cz;
        int64_t e = ex + int64_t(G.nx) * (ey + int64_t(G.ny) * ez);
        if (!mask[e]) continue;
        int pl = ((pi - 2 * ex) >> 1) + 2 * ((pj - 2 * ey) >> 1) + 4 * ((pk - 2 * ez) >> 1);
        int b = (ji - 2 * ex) + 3 * (jj - 2 * ey) + 9 * (jk - 2 * ez);
        for (int q = 0; q < 27; ++q) {
          double f = -T->w[q] * sc * T->psi[q][pl];
          const double* db = T->dphi[q][b];
          out[0] = fma(f, db[0], out[0]);
          out[1] = fma(f, db[1], out[1]);
          out[2] = fma(f, db[2], out[2]);
        }
      }
}

// The same entry for the P1-disc pressure (Section 2's element pair): row P = 4 f + k is the
// k-th basis function (1, xi, eta, zeta) of fluid element f, which alone carries it.
__device__ void divergence_entry_p1(int64_t P, int64_t J, const Geo& G, const int32_t* fluid, const RefTables* T,
                                    double out[3]) {
  const int64_t e = fluid[P >> 2];
  const int k = int(P & 3);
  const int ex = int(e % G.nx), ey = int((e / G.nx) % G.ny), ez = int(e / (int64_t(G.nx) * G.ny));
  int ji, jj, jk;
  node_ijk(J, G, ji, jj, jk);
  const int b = (ji - 2 * ex) + 3 * (jj - 2 * ey) + 9 * (jk - 2 * ez);
  const double sc = 0.25 * G.h * G.h;
  out[0] = out[1] = out[2] = 0.0;
  for (int q = 0; q < 27; ++q) {
    const double f = -T->w[q] * sc * T->p1[q][k];
    const double* db = T->dphi[q][b];
    out[0] = fma(f, db[0], out[0]);
    out[1] = fma(f, db[1], out[1]);
    out[2] = fma(f, db[2], out[2]);
  }
}

// ------------------------------------------------------------------ a2: assembly
// On GB300 a warp-wide FP64 instruction holds the FP64 pipe for the same time whether 1 or 32
// lanes are active, so the assembly is organised for uniform lanes: one thread per work unit
// (an upper block (I, J >= I) and one fluid element holding both nodes), each unit exactly 27
// Gauss points.  Per unit the thread accumulates
//   O[c][d] = sum_q f_q dphi_b,c(q) dphi_a,d(q),   f_q = nu_q w_q (h/2)^3 (2/h)^2,
// and the element's contribution to the block is tr(O) I + O for the symmetric form 2 nu D:D
// (Section 3) and tr(O) I for the gradient form nu grad:grad (Section 2).  A CTA holds the
// units of whole blocks (at most 256); each block sums its units' O in element order in
// shared memory, then writes itself and, off the diagonal, its transpose (operator symmetric).
struct SmemTables {
  double dphi[27][27][3];
  double wsc[27];
};

__global__ void __launch_bounds__(256) k_assemble_A(const int32_t* __restrict__ asm_cta,
                                                    const int32_t* __restrict__ asm_uoff,
                                                    const uint32_t* __restrict__ asm_unit,
                                                    const int32_t* __restrict__ a_tpos,
                                                    const double* __restrict__ nu, const RefTables* __restrict__ T,
                                                    double sc, int form, const double* __restrict__ dn,
                                                    double* __restrict__ val) {
  __shared__ SmemTables st;
  __shared__ double part[256][10];  // per unit: the block's non-trace part, then the trace term
  {
    const double* src = &T->dphi[0][0][0];
    double* dst = &st.dphi[0][0][0];
    for (int e = threadIdx.x; e < 27 * 27 * 3; e += blockDim.x) dst[e] = src[e];
    if (threadIdx.x < 27) st.wsc[threadIdx.x] = T->w[threadIdx.x] * sc;
  }
  __syncthreads();
  const int blk0 = asm_cta[blockIdx.x], blk1 = asm_cta[blockIdx.x + 1];
  const int u0 = asm_uoff[blk0], u1 = asm_uoff[blk1];
  const int u = u0 + int(threadIdx.x);
  double O[9], ON[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) O[c] = ON[c] = 0.0;
  if (u < u1) {
    const uint32_t w = asm_unit[u];
    const int fe = int(w >> 10), a = int((w >> 5) & 31u), b = int(w & 31u);
    const double* nq = nu + int64_t(fe) * 27;
    if (form == GDSW_FORM_SYMMETRIC) {
      for (int q = 0; q < 27; ++q) {
        const double f = __ldg(nq + q) * st.wsc[q];
        const double* da = st.dphi[q][a];
        const double* db = st.dphi[q][b];
        const double fa0 = f * da[0], fa1 = f * da[1], fa2 = f * da[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double dbc = db[c];
          O[c * 3 + 0] = fma(dbc, fa0, O[c * 3 + 0]);
          O[c * 3 + 1] = fma(dbc, fa1, O[c * 3 + 1]);
          O[c * 3 + 2] = fma(dbc, fa2, O[c * 3 + 2]);
        }
      }
      if (dn) {  // Newton term: N (D grad phi_a)_c (D grad phi_b)_d at every Gauss point
        for (int q = 0; q < 27; ++q) {
          const double* g = dn + (int64_t(fe) * 27 + q) * 7;
          const double Dm[3][3] = {{g[0], g[3], g[4]}, {g[3], g[1], g[5]}, {g[4], g[5], g[2]}};
          const double f = g[6] * st.wsc[q];
          const double* da = st.dphi[q][a];
          const double* db = st.dphi[q][b];
          double ga[3], gb[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            ga[c] = Dm[c][0] * da[0] + Dm[c][1] * da[1] + Dm[c][2] * da[2];
            gb[c] = Dm[c][0] * db[0] + Dm[c][1] * db[1] + Dm[c][2] * db[2];
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const double fc = f * ga[c];
#pragma unroll
            for (int d = 0; d < 3; ++d) ON[c * 3 + d] = fma(fc, gb[d], ON[c * 3 + d]);
          }
        }
      }
    } else {  // only the trace is needed
      for (int q = 0; q < 27; ++q) {
        const double f = __ldg(nq + q) * st.wsc[q];
        const double* da = st.dphi[q][a];
        const double* db = st.dphi[q][b];
        O[0] = fma(f * da[0], db[0], O[0]);
        O[4] = fma(f * da[1], db[1], O[4]);
        O[8] = fma(f * da[2], db[2], O[8]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) part[threadIdx.x][c] = form == GDSW_FORM_SYMMETRIC ? O[c] + ON[c] : 0.0;
  part[threadIdx.x][9] = O[0] + O[4] + O[8];
  __syncthreads();
  for (int blk = blk0 + int(threadIdx.x); blk < blk1; blk += blockDim.x) {
    const int v0 = asm_uoff[blk], v1 = asm_uoff[blk + 1];
    if (v1 == v0) continue;  // a lower block: written as the transpose of its upper partner
    double S[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) S[c] = part[v0 - u0][c];
    for (int v = v0 + 1; v < v1; ++v)
#pragma unroll
      for (int c = 0; c < 10; ++c) S[c] += part[v - u0][c];
    const double tr = S[9];
    double out[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) out[c] = S[c];
    out[0] += tr;
    out[4] += tr;
    out[8] += tr;
    double* vp = val + int64_t(blk) * 9;
#pragma unroll
    for (int c = 0; c < 9; ++c) vp[c] = out[c];
    const int tb = a_tpos[blk];
    if (tb != blk) {
      double* wp = val + int64_t(tb) * 9;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) wp[d * 3 + c] = out[c * 3 + d];
    }
  }
}

// pfluid != nullptr: P1-disc rows (fluid element list), else Q1 rows (pressure node list)
__global__ void k_assemble_B(const int32_t* __restrict__ b_ptr, const int32_t* __restrict__ b_col,
                             const int32_t* __restrict__ pnode, const int32_t* __restrict__ pfluid,
                             const int32_t* __restrict__ vnode, int64_t np, Geo G, const uint8_t* mask,
                             const RefTables* T, double* __restrict__ bval) {
  int64_t P = blockIdx.x * int64_t(blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (P >= np) return;
  for (int e = b_ptr[P] + lane; e < b_ptr[P + 1]; e += 32) {
    double out[3];
    if (pfluid)
      divergence_entry_p1(P, vnode[b_col[e]], G, pfluid, T, out);
    else
      divergence_entry(pnode[P], vnode[b_col[e]], G, mask, T, out);
    bval[int64_t(e) * 3 + 0] = out[0];
    bval[int64_t(e) * 3 + 1] = out[1];
    bval[int64_t(e) * 3 + 2] = out[2];
  }
}

__global__ void k_copy_bt(const int32_t* __restrict__ bt2b, int64_t nbt, const double* __restrict__ bval,
                          double* __restrict__ btval) {
  int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= nbt) return;
  int64_t s = bt2b[e];
  btval[e * 3 + 0] = bval[s * 3 + 0];
  btval[e * 3 + 1] = bval[s * 3 + 1];
  btval[e * 3 + 2] = bval[s * 3 + 2];
}

// b = -A_(free, D) g_D.  One warp per row that has a Dirichlet neighbour with g != 0 (the
// rows are listed at set-up; every other entry of b is zero); the lanes take the row's
// Dirichlet neighbours and the warp sums them with a fixed butterfly.
__global__ void __launch_bounds__(256) k_lift(const int32_t* __restrict__ rows, int64_t nrows,
                                              const int32_t* ad_ptr, const int32_t* ad_col, const int32_t* vnode,
                                              int64_t nv, const int32_t* bd_ptr, const int32_t* bd_col,
                                              const int32_t* pnode, const int32_t* pfluid, Geo G,
                                              const uint8_t* mask, const int32_t* felem, const double* nu,
                                              const RefTables* T, int form, const double* g, double* b) {
  const int64_t w = blockIdx.x * int64_t(blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (w >= nrows) return;
  const int64_t row = rows[w];
  if (row < nv) {
    double acc[3] = {0, 0, 0};
    for (int e = ad_ptr[row] + lane; e < ad_ptr[row + 1]; e += 32) {
      int64_t J = ad_col[e];
      double blk[9];
      velocity_block(vnode[row], J, G, mask, felem, nu, T, form, blk);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[c] = fma(blk[c * 3 + d], g[3 * J + d], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane < 3) b[3 * row + lane] = -(lane == 0 ? acc[0] : (lane == 1 ? acc[1] : acc[2]));
  } else {
    const int64_t P = row - nv;
    double acc = 0.0;
    for (int e = bd_ptr[P] + lane; e < bd_ptr[P + 1]; e += 32) {
      int64_t J = bd_col[e];
      double v[3];
      if (pfluid)
        divergence_entry_p1(P, J, G, pfluid, T, v);
      else
        divergence_entry(pnode[P], J, G, mask, T, v);
      acc = fma(v[0], g[3 * J], fma(v[1], g[3 * J + 1], fma(v[2], g[3 * J + 2], acc)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) b[3 * nv + P] = -acc;
  }
}

// ------------------------------------------------------------------ a3: SpMV
// Velocity rows from the sliced copy: slices of 32 rows, lane = row, every lane running the
// same number of blocks (the slice's longest row; shorter rows are zero padded),
// so each FP64 warp instruction has all 32 lanes busy.  Slot group g (32 slots, one per lane)
// keeps its 3x3 blocks component-major: value m of lane l at g * 288 + m * 32 + l (B^T: at
// g * 96 + m * 32 + l), so every value load is one coalesced 256-byte access.
// Pressure rows: one warp per row streaming the contiguous 3-vectors of B.  FP64 throughout;
// y = A x or y = b - A x.
__global__ void k_sell_fill(const int32_t* __restrict__ src, int64_t nslots, int m, const double* __restrict__ from,
                            double* __restrict__ to) {
  const int64_t slot = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (slot >= nslots) return;
  const int64_t g = slot >> 5;
  const int lane = int(slot & 31);
  const int32_t e = src[slot];
  for (int c = 0; c < m; ++c) to[g * (32 * m) + c * 32 + lane] = e >= 0 ? from[int64_t(e) * m + c] : 0.0;
}

__device__ __forceinline__ void sell_block(const int32_t* __restrict__ acol, const double* __restrict__ aval,
                                           const double* __restrict__ x, int64_t g, int lane, double& a0, double& a1,
                                           double& a2) {
  const int64_t j = __ldg(acol + g * 32 + lane);
  const double x0 = __ldg(x + 3 * j), x1 = __ldg(x + 3 * j + 1), x2 = __ldg(x + 3 * j + 2);
  const double* v = aval + g * 288 + lane;
  const double v0 = __ldcs(v), v1 = __ldcs(v + 32), v2 = __ldcs(v + 64), v3 = __ldcs(v + 96), v4 = __ldcs(v + 128),
               v5 = __ldcs(v + 160), v6 = __ldcs(v + 192), v7 = __ldcs(v + 224), v8 = __ldcs(v + 256);
  a0 = fma(v2, x2, fma(v1, x1, fma(v0, x0, a0)));
  a1 = fma(v5, x2, fma(v4, x1, fma(v3, x0, a1)));
  a2 = fma(v8, x2, fma(v7, x1, fma(v6, x0, a2)));
}

// Velocity part: CTA b takes slices 2b and 2b + 1, four warps per slice; warp k of a slice
// takes the slot groups g = g0 + k, g0 + k + 4, ... (two in flight), and the four partial
// sums of a row are added in warp order.  CTAs from ceil(nslices / 2) on take 8 pressure rows.
__global__ void __launch_bounds__(256) k_spmv(const int32_t* __restrict__ sell_row, const int64_t* __restrict__ aoff,
                                              const int32_t* __restrict__ acol, const double* __restrict__ aval,
                                              const int64_t* __restrict__ boff, const int32_t* __restrict__ bcol,
                                              const double* __restrict__ btval, int64_t nslices,
                                              const int32_t* __restrict__ b_ptr, const int32_t* __restrict__ b_col,
                                              const double* __restrict__ bval, int64_t nv, int64_t np,
                                              const double* __restrict__ x, double* __restrict__ y,
                                              const double* __restrict__ rhs) {
  __shared__ double red[8][3][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nu = 3 * nv;
  const int64_t vblocks = (nslices + 1) / 2;
  // launched in plain stream order (chained, it measured slower than the launch latency it
  // hid); it lets its chained successor start early
  dep_release();
  if (blockIdx.x < vblocks) {
    const int64_t sl = 2 * int64_t(blockIdx.x) + (warp >> 2);
    const int sub = warp & 3;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    if (sl < nslices) {
      const int64_t g0 = aoff[sl] >> 5, g1 = aoff[sl + 1] >> 5;
      int64_t g = g0 + sub;
      // two slot groups per pass, their loads independent of the accumulators (so both are in
      // flight at once) and their products chained into the same three sums: no extra FP64
      // adds to merge partial sums, since the FP64 pipe, not memory, bounds this loop
      for (; g + 4 < g1; g += 8) {
        const int64_t j = __ldg(acol + g * 32 + lane), k = __ldg(acol + (g + 4) * 32 + lane);
        const double* v = aval + g * 288 + lane;
        const double* w = aval + (g + 4) * 288 + lane;
        double vv[9], ww[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          vv[q] = __ldcs(v + 32 * q);
          ww[q] = __ldcs(w + 32 * q);
        }
        const double x0 = __ldg(x + 3 * j), x1 = __ldg(x + 3 * j + 1), x2 = __ldg(x + 3 * j + 2);
        const double y0 = __ldg(x + 3 * k), y1 = __ldg(x + 3 * k + 1), y2 = __ldg(x + 3 * k + 2);
        a0 = fma(vv[2], x2, fma(vv[1], x1, fma(vv[0], x0, a0)));
        a1 = fma(vv[5], x2, fma(vv[4], x1, fma(vv[3], x0, a1)));
        a2 = fma(vv[8], x2, fma(vv[7], x1, fma(vv[6], x0, a2)));
        a0 = fma(ww[2], y2, fma(ww[1], y1, fma(ww[0], y0, a0)));
        a1 = fma(ww[5], y2, fma(ww[4], y1, fma(ww[3], y0, a1)));
        a2 = fma(ww[8], y2, fma(ww[7], y1, fma(ww[6], y0, a2)));
      }
      if (g < g1) sell_block(acol, aval, x, g, lane, a0, a1, a2);
      const int64_t h0 = boff[sl] >> 5, h1 = boff[sl + 1] >> 5;
      for (int64_t h = h0 + sub; h < h1; h += 4) {
        const double xp = __ldg(x + nu + __ldg(bcol + h * 32 + lane));
        const double* v = btval + h * 96 + lane;
        a0 = fma(__ldcs(v + 0), xp, a0);
        a1 = fma(__ldcs(v + 32), xp, a1);
        a2 = fma(__ldcs(v + 64), xp, a2);
      }
    }
    red[warp][0][lane] = a0;
    red[warp][1][lane] = a1;
    red[warp][2][lane] = a2;
    __syncthreads();
    if (sub == 0 && sl < nslices) {
      const int32_t row = sell_row[sl * 32 + lane];
      if (row >= 0) {
        const int64_t o = 3 * int64_t(row);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double t = red[warp][c][lane];
#pragma unroll
          for (int k = 1; k < 4; ++k) t += red[warp + k][c][lane];
          y[o + c] = rhs ? rhs[o + c] - t : t;
        }
      }
    }
  } else {
    const int64_t P = (int64_t(blockIdx.x) - vblocks) * 8 + warp;
    if (P >= np) return;
    const int64_t f0 = int64_t(b_ptr[P]) * 3, f1 = int64_t(b_ptr[P + 1]) * 3;
    double acc = 0.0;
    for (int64_t f = f0 + lane; f < f1; f += 32) {
      const int64_t e = f / 3;
      const int d = int(f - 3 * e);
      acc = fma(__ldcs(bval + f), __ldg(x + 3 * int64_t(b_col[e]) + d), acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[nu + P] = rhs ? rhs[nu + P] - acc : acc;
  }
}

// ------------------------------------------------------------------ launchers
static Geo geo(const gdsw_ctx* c) {
  Geo G;
  G.nx = c->mesh.nx; G.ny = c->mesh.ny; G.nz = c->mesh.nz;
  G.NX = c->mesh.NX; G.NY = c->mesh.NY;
  G.h = c->mesh.h;
  return G;
}

void upload_tables(gdsw_ctx* c, cudaStream_t s) {
  RefTables T;
  host_tables(T);
  RefTables* d = c->arena.alloc<RefTables>(1);
  GDSW_CUDA(cudaMemcpyAsync(d, &T, sizeof(T), cudaMemcpyHostToDevice, s));
  GDSW_CUDA(cudaStreamSynchronize(s));
  c->d_tables = d;
}

// Picard update (Section 3): u_k at every free velocity node from the solution x (free dofs in
// solve order); the Dirichlet nodes keep their data g (copied before this kernel)
__global__ void k_picard_velocity(const int32_t* __restrict__ vnode, int64_t nv, const double* __restrict__ x,
                                  double* __restrict__ uk) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= 3 * nv) return;
  const int64_t I = q / 3;
  uk[3 * int64_t(vnode[I]) + (q - 3 * I)] = x[q];
}

__global__ void k_axpy(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) x[i] += d[i];
}

void launch_axpy(double* x, const double* d, int64_t n, cudaStream_t s) {
  if (n == 0) return;
  k_axpy<<<int((n + 255) / 256), 256, 0, s>>>(x, d, n);
  check_launch("k_axpy");
}

void launch_picard_velocity(gdsw_ctx* c, const double* x, cudaStream_t s) {
  const int64_t nv = c->mesh.nv;
  GDSW_CUDA(cudaMemcpyAsync(c->d_uk, c->d_gdir, sizeof(double) * 3 * c->mesh.nnodes, cudaMemcpyDeviceToDevice, s));
  if (nv > 0) {
    k_picard_velocity<<<int((3 * nv + 255) / 256), 256, 0, s>>>(c->d_vnode, nv, x, c->d_uk);
    check_launch("k_picard_velocity");
  }
  c->has_uk = true;
}

void launch_viscosity(gdsw_ctx* c, cudaStream_t s) {
  int64_t nfe = int64_t(c->mesh.fluid.size());
  int64_t n = nfe * 27;
  k_viscosity<<<int((n + 255) / 256), 256, 0, s>>>(c->d_fluid, nfe, c->d_uk, static_cast<RefTables*>(c->d_tables),
                                                  geo(c), c->form, c->has_uk ? 1 : 0, c->nu0, c->nu_inf, c->lam,
                                                  c->ncar, c->d_nu, c->d_dn);
  check_launch("k_viscosity");
}

void launch_assembly(gdsw_ctx* c, cudaStream_t s, bool newton) {
  const auto* T = static_cast<RefTables*>(c->d_tables);
  const int64_t np = c->mesh.np;
  double* aval = c->d_val;
  double* btval = c->d_val + 9 * c->nnzb;
  double* bval = btval + 3 * c->nbt;
  const int ncta = int(c->mesh.asm_cta.size()) - 1;
  if (ncta > 0)
    k_assemble_A<<<ncta, 256, 0, s>>>(c->d_asm_cta, c->d_asm_uoff, c->d_asm_unit, c->d_a_tpos, c->d_nu, T,
                                      0.5 * c->mesh.h, c->form, newton ? c->d_dn : nullptr, aval);
  check_launch("k_assemble_A");
  if (c->b_assembled) {  // B = -(q, div u) depends on the mesh only, not on the viscosity
    launch_sell_fill(c, false, s);
    return;
  }
  k_assemble_B<<<int((np + 7) / 8), 256, 0, s>>>(c->d_b_ptr, c->d_b_col, c->d_pnode,
                                                 c->mesh.pdisc ? c->d_fluid : nullptr, c->d_vnode, np, geo(c),
                                                 c->d_mask, T, bval);
  check_launch("k_assemble_B");
  if (c->nbt > 0) {
    k_copy_bt<<<int((c->nbt + 255) / 256), 256, 0, s>>>(c->d_bt2b, c->nbt, bval, btval);
    check_launch("k_copy_bt");
  }
  launch_sell_fill(c, true, s);
  c->b_assembled = true;
}

void launch_lift(gdsw_ctx* c, double* b, cudaStream_t s) {
  int64_t nv = c->mesh.nv, np = c->mesh.np;
  // every entry of b not written below (rows without a Dirichlet neighbour) is zero
  GDSW_CUDA(cudaMemsetAsync(b, 0, size_t(3 * nv + np) * sizeof(double), s));
  if (c->n_lift_rows == 0) return;
  k_lift<<<int((c->n_lift_rows + 7) / 8), 256, 0, s>>>(c->d_lift_rows, c->n_lift_rows, c->d_ad_ptr, c->d_ad_col,
                                                       c->d_vnode, nv, c->d_bd_ptr, c->d_bd_col, c->d_pnode,
                                                       c->mesh.pdisc ? c->d_fluid : nullptr, geo(c),
                                                       c->d_mask, c->d_felem, c->d_nu,
                                                       static_cast<RefTables*>(c->d_tables), c->form, c->d_gdir, b);
  check_launch("k_lift");
}

void launch_spmv(gdsw_ctx* c, const double* x, double* y, const double* rhs, cudaStream_t s) {
  const int64_t nv = c->mesh.nv, np = c->mesh.np;
  const double* bval = c->d_val + 9 * c->nnzb + 3 * c->nbt;
  const int64_t ns = c->n_sell_slices;
  const int64_t blocks = (ns + 1) / 2 + (np + 7) / 8;
  k_spmv<<<int(blocks), 256, 0, s>>>(c->d_sell_row, c->d_sell_aoff, c->d_sell_acol, c->d_sell_aval,
                                     c->d_sell_boff, c->d_sell_bcol, c->d_sell_btval, ns, c->d_b_ptr, c->d_b_col,
                                     bval, nv, np, x, y, rhs);
  check_launch("k_spmv");
}

// refresh the sliced copy of A (after every assembly) and of B^T (once B is assembled)
void launch_sell_fill(gdsw_ctx* c, bool with_bt, cudaStream_t s) {
  const MeshHost& M = c->mesh;
  const int64_t na = int64_t(M.sell_acol.size()), nb = int64_t(M.sell_bcol.size());
  if (na > 0) {
    k_sell_fill<<<int((na + 255) / 256), 256, 0, s>>>(c->d_sell_asrc, na, 9, c->d_val, c->d_sell_aval);
    check_launch("k_sell_fill");
  }
  if (with_bt && nb > 0) {
    k_sell_fill<<<int((nb + 255) / 256), 256, 0, s>>>(c->d_sell_bsrc, nb, 3, c->d_val + 9 * c->nnzb,
                                                      c->d_sell_btval);
    check_launch("k_sell_fill");
  }
}

}  // namespace gdsw
