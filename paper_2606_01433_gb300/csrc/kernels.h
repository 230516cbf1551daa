// Declarations of the kernel launchers shared between translation units.
#pragma once

#include "common.h"

namespace gdsw {

struct GemmTaskP {
  const void* a;
  const void* b;
  void* c;
  int32_t M, N, K, lda, ldb, ldc;
  int32_t ta, tb;
  double alpha, beta;
};

struct InvTaskP {
  void* a;
  int32_t n, ld;
  int32_t id;
};

// Q2 / Q1 reference tables at the 27 Gauss points (host computed, device resident)
struct RefTables {
  double dphi[27][27][3];   // [q][a][l]
  double psi[27][8];        // [q][P]
  double p1[27][4];         // [q][k]: P1-disc basis 1, xi, eta, zeta
  double w[27];
};
void host_tables(RefTables& T);

// dense.cu
template <typename TM, typename TV>
void launch_gemv(const TM* M, const TV* x, TV* y, const TV* b, const GemvPlan& P, int launch, int max_ld,
                 cudaStream_t s);
void set_gemv_smem_limits();
template <typename TM, typename TV>
void size_sweep(SweepPlan& P);
template <typename TM, typename TV>
void launch_sweep(const TM* M, TV* vec, const SweepPlan& P, unsigned* flag, int T, cudaStream_t s);
template <typename TV>
void launch_sym_reduce(const TV* vec, TV* y, const GemvPlan& P, int T, cudaStream_t s);
struct PackTile {
  int64_t src, dst;
  int32_t ld, rows, cols, pad;  // rows/cols valid inside the tile
};
template <typename T>
void pack_tiles(DevArena& tmp, const T* src, T* dst, const std::vector<PackTile>& tiles, int TT, cudaStream_t s);
// tile edge of the packed symmetric blocks: one 16-byte load per lane across a warp
inline int sym_tile_size(int prec) { return prec == GDSW_FP64 ? 64 : (prec == GDSW_FP32 ? 128 : 256); }
// column tile of the transposed GEMV: 16 lanes (half a warp) x one 16-byte load of entries
inline int gemvt_tile_cols(int prec) { return prec == GDSW_FP64 ? 32 : (prec == GDSW_FP32 ? 64 : 128); }
template <typename T>
void run_gemm(DevArena& tmp, const std::vector<GemmTaskP>& tasks, cudaStream_t s);
template <typename T>
void run_gemm_engine(DevArena& tmp, const std::vector<GemmTaskP>& tasks, cudaStream_t s, int engine);
void set_gemm_engine(int e);
int gemm_engine();
// tc_gemm.cu: FP32 tasks on the tensor cores (3xTF32); synchronises the stream
void run_gemm_tc(const std::vector<GemmTaskP>& tasks, cudaStream_t s);
template <typename T>
void run_inverse(DevArena& tmp, const std::vector<InvTaskP>& tasks, std::vector<double>& minpiv, cudaStream_t s);
void convert(const void* src, int sprec, void* dst, int dprec, int64_t n, cudaStream_t s);

// operator.cu
void launch_viscosity(gdsw_ctx* c, cudaStream_t s);
void launch_picard_velocity(gdsw_ctx* c, const double* x, cudaStream_t s);
void launch_axpy(double* x, const double* d, int64_t n, cudaStream_t s);  // x += d
// newton: add the Newton term from the D(u_k), N values of the last viscosity launch (d_dn)
void launch_assembly(gdsw_ctx* c, cudaStream_t s, bool newton = false);
void launch_lift(gdsw_ctx* c, double* b, cudaStream_t s);
void launch_spmv(gdsw_ctx* c, const double* x, double* y, const double* b, cudaStream_t s);
void launch_sell_fill(gdsw_ctx* c, bool with_bt, cudaStream_t s);
void upload_tables(gdsw_ctx* c, cudaStream_t s);

// schwarz.cu
struct ProMeta {
  int64_t phi, ioff, coff;
  int32_t ld, nI, c, pad;
};
template <typename TV>
void launch_gather(const double* r, const int32_t* idx, TV* out, int64_t n, cudaStream_t s);
template <typename TV>
void launch_scatter(const TV* x, const int32_t* ptr, const int32_t* pos, const double* w, double* z, int n,
                    int accumulate, cudaStream_t s);
void launch_restrict(const LevelDev& L, const double* r, double* r0, cudaStream_t s);
void launch_prolong(const LevelDev& L, const double* x0, double* z, cudaStream_t s);
void launch_axpy_gamma(const int32_t* gu_dof, const int32_t* gu_ptr, const int32_t* gcol, const double* gval,
                       int64_t ngu, const double* x0, double* z, cudaStream_t s);

}  // namespace gdsw
